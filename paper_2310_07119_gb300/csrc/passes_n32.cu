// FP32 line passes of length 32.
#define TWA_N 32
#include "passes_inst.inc"
