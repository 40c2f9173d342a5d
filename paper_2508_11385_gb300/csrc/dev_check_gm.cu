// dev_check_gm.cu -- build-time check of the kernels that write a general
// output (COOT_GM bit 8: an output whose rows are not adjacent, such as the
// transposed output of a cumsum along dim 0 scanned over the transposed
// problem).  Like dev_check.cu, the object is not linked into the library.
#define COOT_GM 256
#include "coot_kernels.cuh"
using namespace coot;

// Y = 0.5*A + B % exp(C)
typedef eGlue<eOp<Leaf<0>, eop_scalar_times<0>>, eGlue<Leaf<1>, eOp<Leaf<2>, eop_exp>, eglue_schur>, eglue_plus> T3;
// A % B
typedef eGlue<Leaf<0>, Leaf<1>, eglue_schur> T2;

#define KB(name, bound, minb, body) \
  extern "C" __global__ void __launch_bounds__(bound, minb) name(const __grid_constant__ Params p) { body(p); }

// one-pass row scans with transposed slots (TRMASK) and a transposed output
KB(chk_scanp_tr_f32, 256, 2, (scanp_kernel<T3, float, 3, 1, 1, 16, 8, 5>))
KB(chk_scanp_tr_bf16, 256, 2, (scanp_kernel<T3, bf16, 3, 1, 1, 16, 8, 2>))
KB(chk_scanp_tr_f64, 256, 2, (scanp_kernel<T3, double, 3, 1, 1, 16, 8, 7>))
KB(chk_scanp_tr_i32, 256, 2, (scanp_kernel<T2, int, 2, 0, 1, 16, 8, 1>))
KB(chk_scanp_gm_f32, 256, 2, (scanp_kernel<T3, float, 3, 1, 1, 16, 8, 0>))
