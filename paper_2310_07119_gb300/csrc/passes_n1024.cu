// FP32 line passes of length 1024.
#define TWA_N 1024
#include "passes_inst.inc"
