// Piecewise-linear block engine, mixed (FP32 regular pairs) form.
#define BEM_P1_MIXED 1
#include "bem_block_p1.inl"
