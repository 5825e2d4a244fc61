// FP32 line passes of length 16.
#define TWA_N 16
#include "passes_inst.inc"
