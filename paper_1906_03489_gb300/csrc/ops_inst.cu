// One instantiation unit of the operator kernel: compiled once per
// (precision, dimension, operator) with -DSPX_TN=f32|f64 -DSPX_DIM=2|3 -DSPX_OP=0..5.
#include "launch_ops.cuh"

#ifndef SPX_TN
#error "compile with -DSPX_TN=f32|f64 -DSPX_DIM=2|3 -DSPX_OP=0..5"
#endif

#define SPX_CAT2_(a, b) a##b
#define SPX_CAT2(a, b) SPX_CAT2_(a, b)
#define SPX_T_f32 float
#define SPX_T_f64 double
#define SPX_TYPE(tn) SPX_CAT2(SPX_T_, tn)

SPX_DEFINE_LAUNCH(SPX_TN, SPX_TYPE(SPX_TN), SPX_DIM, SPX_OP)
