// Piecewise-linear block engine, FP64 form.
#define BEM_P1_MIXED 0
#include "bem_block_p1.inl"
