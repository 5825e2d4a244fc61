// FP32 line passes of length 128.
#define TWA_N 128
#include "passes_inst.inc"
