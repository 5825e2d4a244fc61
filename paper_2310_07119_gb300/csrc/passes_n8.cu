// FP32 line passes of length 8.
#define TWA_N 8
#include "passes_inst.inc"
