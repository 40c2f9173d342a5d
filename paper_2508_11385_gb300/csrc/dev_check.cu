// dev_check.cu -- build-time check of the device expression templates.
//
// The kernels of this library are generated per expression tree and compiled
// by NVRTC at run time.  This translation unit instantiates every kernel
// family once for representative trees and storage types with nvcc for
// sm_103a, so that an error in the device headers fails the build, and the
// build log records registers and shared memory per family (-Xptxas -v).
// The object is not linked into the library.
#include "coot_kernels.cuh"
using namespace coot;

// Y = 0.5*A + B % exp(C)
typedef eGlue<eOp<Leaf<0>, eop_scalar_times<0>>, eGlue<Leaf<1>, eOp<Leaf<2>, eop_exp>, eglue_schur>, eglue_plus> T3;
// A % B
typedef eGlue<Leaf<0>, Leaf<1>, eglue_schur> T2;
// sqrt(abs(exp(A-B) / (1 + abs(C)) % D - E)) % F
typedef eGlue<eOp<eOp<eGlue<eGlue<eOp<eGlue<Leaf<0>, Leaf<1>, eglue_minus>, eop_exp>,
                                  eOp<eOp<Leaf<2>, eop_abs>, eop_scalar_plus<0>>, eglue_div>,
                            Leaf<3>, eglue_schur>, eop_abs>, eop_sqrt>, Leaf<5>, eglue_schur> T6;

#define K(name, bound, body) \
  extern "C" __global__ void __launch_bounds__(bound) name(const __grid_constant__ Params p) { body(p); }
// the tile family with the register caps its generated kernels use
#define KB(name, bound, minb, body) \
  extern "C" __global__ void __launch_bounds__(bound, minb) name(const __grid_constant__ Params p) { body(p); }

K(chk_str_f32, 512, (str_kernel<T3, float, 3, 1, RED_SUM, 4, 2, true>))
K(chk_str_bf16, 512, (str_kernel<T3, bf16, 3, 1, RED_SSQ, 8, 1, true>))
K(chk_str_f16_var, 512, (str_kernel<T3, f16, 3, 1, RED_CSQ, 8, 2, false>))
K(chk_str_f64, 512, (str_kernel<T3, double, 3, 1, RED_CSQ, 2, 2, false>))
K(chk_str_i32_dot, 512, (str_kernel<T2, int, 2, 0, RED_DOT, 4, 2, true>))
K(chk_str_l8, 512, (str_kernel<T6, float, 6, 1, RED_NONE, 4, 2, true>))
K(chk_col_f32, 512, (col_kernel<T3, float, 3, 1, RED_SUM, 4, 2, true>))
K(chk_row_f16, 512, (row_kernel<T3, f16, 3, 1, RED_SUM, 8, 2, true>))
KB(chk_tile_dim0, 256, 4, (tile_kernel<T3, float, 3, 1, RED_SUM, 0, 4, true>))
KB(chk_tile_dim1, 256, 4, (tile_kernel<T3, float, 3, 1, RED_SUM, 1, 5, true>))
KB(chk_tile_f64, 256, 4, (tile_kernel<T3, double, 3, 1, RED_MEAN1, -1, 1, false>))
K(chk_adj_f32, 512, (adj_kernel<T3, float, 3, 1, 4, 2>))
extern "C" __global__ void __launch_bounds__(256) chk_batch(const __grid_constant__ BatchParams p) {
  batch_kernel<T3, float, 3, 1, 4, true>(p);
}
extern "C" __global__ void __launch_bounds__(BATCHF_THREADS, 5) chk_batchf(const __grid_constant__ BatchParams p) {
  batchf_kernel<T3, float, 3, 1, 4, true, 8192>(p);
}
extern "C" __global__ void __launch_bounds__(BATCHF_THREADS, 5) chk_batchf_f64_2tr(const __grid_constant__ BatchParams p) {
  batchf_kernel<eGlue<Leaf<0>, Leaf<1>, eglue_plus>, double, 2, 0, 3, true, 2560>(p);
}
extern "C" __global__ void __launch_bounds__(256) chk_batch_f64_2tr(const __grid_constant__ BatchParams p) {
  batch_kernel<eGlue<Leaf<0>, Leaf<1>, eglue_plus>, double, 2, 0, 3, true>(p);
}
extern "C" __global__ void __launch_bounds__(256) chk_batch_f32_2tr(const __grid_constant__ BatchParams p) {
  batch_kernel<eGlue<Leaf<0>, Leaf<1>, eglue_plus>, float, 2, 0, 3, false>(p);
}
KB(chk_tilev_f32, 256, 3, (tilev_kernel<T3, float, 3, 1, RED_NONE, -1, 4, true, 4>))
KB(chk_tilev_bf16, 256, 2, (tilev_kernel<T3, bf16, 3, 1, RED_SUM, -1, 4, true, 8>))
KB(chk_tilev_f64, 256, 3, (tilev_kernel<T3, double, 3, 1, RED_CSQ, -1, 4, false, 2>))
// statistics: extremes with positions, products, var along a dim
K(chk_str_imin_f32, 512, (str_kernel<T3, float, 3, 1, RED_IMIN, 4, 2, false>))
K(chk_str_max_bf16, 512, (str_kernel<T3, bf16, 3, 1, RED_MAX, 8, 1, false>))
K(chk_str_prod_f32, 512, (str_kernel<T3, float, 3, 1, RED_PROD, 4, 2, false>))
K(chk_str_prod_f64, 512, (str_kernel<T3, double, 3, 1, RED_PROD, 2, 2, false>))
K(chk_str_prod_i32, 512, (str_kernel<T2, int, 2, 0, RED_PROD, 4, 2, false>))
K(chk_col_min_i32, 512, (col_kernel<T2, int, 2, 0, RED_MIN, 4, 2, false>))
K(chk_col_csq_f32, 512, (col_kernel<T3, float, 3, 1, RED_CSQ, 4, 2, true>))
K(chk_row_imax_f64, 512, (row_kernel<T3, double, 3, 1, RED_IMAX, 2, 2, false>))
K(chk_row_csq_f32, 512, (row_kernel<T3, float, 3, 1, RED_CSQ, 4, 2, false>))
K(chk_row_tr_f32, 512, (row_kernel<T3, float, 3, 1, RED_SUM, 1, 16, false, 5>))
K(chk_row_tr_bf16, 512, (row_kernel<T3, bf16, 3, 1, RED_MAX, 1, 8, false, 2>))
K(chk_row_tr_prod_f64, 512, (row_kernel<T3, double, 3, 1, RED_PROD, 1, 16, false, 1>))
KB(chk_tile_imin_dim0, 256, 4, (tile_kernel<T3, float, 3, 1, RED_IMIN, 0, 4, false>))
KB(chk_tile_csq_dim1, 256, 4, (tile_kernel<T3, double, 3, 1, RED_CSQ, 1, 5, false>))
KB(chk_tilev_prod_f32, 256, 3, (tilev_kernel<T3, float, 3, 1, RED_PROD, -1, 4, false, 4>))
KB(chk_tilev_dim0_f32, 256, 3, (tilev_kernel<T3, float, 3, 1, RED_SUM, 0, 4, true, 4>))
KB(chk_tilev_dim1_bf16, 256, 2, (tilev_kernel<T3, bf16, 3, 1, RED_IMAX, 1, 4, false, 8>))
KB(chk_tilev_dim1_f64, 256, 3, (tilev_kernel<T3, double, 3, 1, RED_CSQ, 1, 4, false, 2>))
// cumsum scans
K(chk_scan_col_f32, 256, (scan_col_kernel<T3, float, 3, 1, 4, 2>))
K(chk_scan_col_t_f64, 256, (scan_col_kernel<T3, double, 3, 1, 2, 1>))
K(chk_scan_col_i32, 256, (scan_col_kernel<T2, int, 2, 0, 4, 2>))
K(chk_scan_row_bf16, 256, (scan_row_kernel<T3, bf16, 3, 1, 8, 2, 2>))
K(chk_scan_row_t_f32, 256, (scan_row_kernel<T3, float, 3, 1, 4, 4, 1>))
KB(chk_scanp_f32, 256, 2, (scanp_kernel<T3, float, 3, 1, 1, 16, 8>))
K(chk_scanp_bf16, 256, (scanp_kernel<T3, bf16, 3, 1, 2, 8, 8>))
K(chk_scanp_f64, 256, (scanp_kernel<T3, double, 3, 1, 2, 8, 8>))
KB(chk_scanp_i32, 256, 2, (scanp_kernel<T2, int, 2, 0, 1, 16, 8>))
// GEMM with a fused epilogue: 2 * P + C (P the product, slot 0), every operand layout
#include "coot_gemm.cuh"
typedef eGlue<eOp<Leaf<0>, eop_scalar_times<0>>, Leaf<1>, eglue_plus> TG;
#define KG(name, body) \
  extern "C" __global__ void __launch_bounds__(256, 2) name(const __grid_constant__ GemmParams p) { body(p); }
KG(chk_gemm_bf16_kk, (gemm_kernel<TG, bf16, 2, 1, 0, true, true>))
KG(chk_gemm_bf16_mn, (gemm_kernel<TG, bf16, 2, 1, 0, false, false>))
KG(chk_gemm_f16_km, (gemm_kernel<TG, f16, 2, 1, 0, true, false>))
KG(chk_gemm_bf16_mk, (gemm_kernel<Leaf<0>, bf16, 1, 0, 0, false, true>))
#define KT(name, body) \
  extern "C" __global__ void __launch_bounds__(GEMM_TC_THREADS, 1) name(const __grid_constant__ GemmParams p) { body(p); }
KT(chk_gemm_tc_bf16_kk, (gemm_tc_kernel<TG, bf16, 2, 1, 0, true, true>))
KT(chk_gemm_tc_f16_kk, (gemm_tc_kernel<Leaf<0>, f16, 1, 0, 0, true, true>))
KT(chk_gemm_tc_bf16_mn, (gemm_tc_kernel<TG, bf16, 2, 1, 0, false, false>))
KT(chk_gemm_tc_bf16_km, (gemm_tc_kernel<Leaf<0>, bf16, 1, 0, 0, true, false>))
#define KS(name, body) \
  extern "C" __global__ void __launch_bounds__(256, 2) name(const __grid_constant__ GemmParams p) { body(p); }
KS(chk_gemm_simt_f32_kk, (gemm_simt_kernel<TG, float, 2, 1, 0, true, true>))
KS(chk_gemm_simt_f32_mn, (gemm_simt_kernel<Leaf<0>, float, 1, 0, 0, false, false>))
KS(chk_gemm_simt_f64_km, (gemm_simt_kernel<TG, double, 2, 1, 0, true, false>))
