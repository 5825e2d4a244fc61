// FP32 line passes of length 2048.
#define TWA_N 2048
#include "passes_inst.inc"
