// One instantiation unit of the operator kernel: compiled once per
// (precision, dimension, operator) with -DSPX_TN=f32|f64 -DSPX_DIM=2|3 -DSPX_OP=0..7,
// and for the 3D Helmholtz of the other basis kinds with -DSPX_TN=.. -DSPX_BK=1|2.
#include "launch_ops.cuh"

#ifndef SPX_TN
#error "compile with -DSPX_TN=f32|f64 -DSPX_DIM=2|3 -DSPX_OP=0..7 (or -DSPX_TN=.. -DSPX_BK=1|2)"
#endif

#define SPX_CAT2_(a, b) a##b
#define SPX_CAT2(a, b) SPX_CAT2_(a, b)
#define SPX_T_f32 float
#define SPX_T_f64 double
#define SPX_TYPE(tn) SPX_CAT2(SPX_T_, tn)

#ifdef SPX_BK
SPX_DEFINE_LAUNCH_BK(SPX_TN, SPX_TYPE(SPX_TN), SPX_BK)
#else
SPX_DEFINE_LAUNCH(SPX_TN, SPX_TYPE(SPX_TN), SPX_DIM, SPX_OP)
#endif
