// FP32 line passes of length 64.
#define TWA_N 64
#include "passes_inst.inc"
