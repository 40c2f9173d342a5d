// coot_dev.cuh -- device-side expression templates of cootgb.
//
// This header is compiled by NVRTC (sm_103a) together with a few generated
// lines that spell one expression tree as a C++ type, e.g.
//     eGlue< eOp<Leaf<0>, eop_scalar_times<0>>,
//            eGlue<Leaf<1>, eOp<Leaf<2>, eop_exp>, eglue_schur>, eglue_plus >
// mirroring the paper's expression classes (Sec. 3): Op<T1,op_type> (trans --
// resolved on the host into the leaf access pattern), eOp<T1,eop_type>
// (element-wise unary, including the scalar forms) and
// eGlue<T1,T2,eglue_type> (element-wise binary).  Like those classes, the
// node types hold no data: an element is evaluated from the values of the
// tree's leaf reads, which the kernel has already loaded into registers, so
// a whole tree costs one load per distinct operand element and no temporary.
//
// Arithmetic per node is IEEE round-to-nearest in the compute type (FP32 for
// FP32/BF16/FP16 storage, FP64 for FP64, wrapping int32 for INT32) with no
// contraction into FMA, so the fused result equals the one-op-at-a-time
// result bit for bit.
#pragma once
#include "coot_params.h"

namespace coot {

typedef long long i64;
typedef unsigned long long u64;
typedef unsigned int u32;
typedef unsigned short u16;

#define COOT_INT_MIN (-2147483647 - 1)

// ---------------------------------------------------------------------------
// storage types and their compute types
// ---------------------------------------------------------------------------
struct bf16 { u16 x; };
struct f16 { u16 x; };

template <class S> struct ctype { typedef S type; };
template <> struct ctype<bf16> { typedef float type; };
template <> struct ctype<f16> { typedef float type; };

// accumulation type of a reduction result
template <class C> struct rtype { typedef C type; };
template <> struct rtype<int> { typedef i64 type; };

template <class C> struct is_int_c { static constexpr bool value = false; };
template <> struct is_int_c<int> { static constexpr bool value = true; };
template <class C> struct is_f32_c { static constexpr bool value = false; };
template <> struct is_f32_c<float> { static constexpr bool value = true; };

// ---------------------------------------------------------------------------
// element conversion between 32-bit words and values
// ---------------------------------------------------------------------------
__device__ __forceinline__ float bf16_lo(u32 w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf16_hi(u32 w) { return __uint_as_float(w & 0xffff0000u); }
__device__ __forceinline__ float f16_to_f32(u16 h) {
  float f;
  asm("cvt.f32.f16 %0, %1;" : "=f"(f) : "h"(h));
  return f;
}
__device__ __forceinline__ u32 pack_bf16x2(float lo, float hi) {
  u32 w;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(w) : "f"(hi), "f"(lo));
  return w;
}
__device__ __forceinline__ u32 pack_f16x2(float lo, float hi) {
  u32 w;
  asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(w) : "f"(hi), "f"(lo));
  return w;
}
__device__ __forceinline__ u16 to_bf16(float v) {
  u16 h;
  asm("cvt.rn.bf16.f32 %0, %1;" : "=h"(h) : "f"(v));
  return h;
}
__device__ __forceinline__ u16 to_f16(float v) {
  u16 h;
  asm("cvt.rn.f16.f32 %0, %1;" : "=h"(h) : "f"(v));
  return h;
}

// raw global loads through the read-only path; stores plain
__device__ __forceinline__ void ldg_words(const void* p, u32 (&w)[4]) {
  asm("ld.global.nc.v4.u32 {%0,%1,%2,%3}, [%4];"
      : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3]) : "l"(p));
}
__device__ __forceinline__ void ldg_words(const void* p, u32 (&w)[2]) {
  asm("ld.global.nc.v2.u32 {%0,%1}, [%2];" : "=r"(w[0]), "=r"(w[1]) : "l"(p));
}
__device__ __forceinline__ void ldg_words(const void* p, u32 (&w)[1]) {
  asm("ld.global.nc.u32 %0, [%1];" : "=r"(w[0]) : "l"(p));
}
__device__ __forceinline__ u16 ldg_u16(const void* p) {
  u16 h;
  asm("ld.global.nc.u16 %0, [%1];" : "=h"(h) : "l"(p));
  return h;
}
__device__ __forceinline__ void stg_words(void* p, const u32 (&w)[4]) {
  asm volatile("st.global.v4.u32 [%0], {%1,%2,%3,%4};" ::"l"(p), "r"(w[0]), "r"(w[1]), "r"(w[2]), "r"(w[3])
               : "memory");
}
__device__ __forceinline__ void stg_words(void* p, const u32 (&w)[2]) {
  asm volatile("st.global.v2.u32 [%0], {%1,%2};" ::"l"(p), "r"(w[0]), "r"(w[1]) : "memory");
}
__device__ __forceinline__ void stg_words(void* p, const u32 (&w)[1]) {
  asm volatile("st.global.u32 [%0], %1;" ::"l"(p), "r"(w[0]) : "memory");
}
__device__ __forceinline__ void stg_u16(void* p, u16 h) {
  asm volatile("st.global.u16 [%0], %1;" ::"l"(p), "h"(h) : "memory");
}

// IO<S>: load/store V consecutive elements (V * sizeof(S) in {2,4,8,16},
// address aligned to that size) or a single element.
template <class S> struct IO;

template <> struct IO<float> {
  typedef float C;
  template <int V> __device__ static void load(const float* p, C (&v)[V]) {
    u32 w[V];
    ldg_words(p, w);
#pragma unroll
    for (int l = 0; l < V; ++l) v[l] = __uint_as_float(w[l]);
  }
  __device__ static C load1(const float* p) {
    u32 w[1];
    ldg_words(p, w);
    return __uint_as_float(w[0]);
  }
  template <int V> __device__ static void store(float* p, const C (&v)[V]) {
    u32 w[V];
#pragma unroll
    for (int l = 0; l < V; ++l) w[l] = __float_as_uint(v[l]);
    stg_words(p, w);
  }
  __device__ static void store1(float* p, C v) {
    u32 w[1] = {__float_as_uint(v)};
    stg_words(p, w);
  }
};

template <> struct IO<int> {
  typedef int C;
  template <int V> __device__ static void load(const int* p, C (&v)[V]) {
    u32 w[V];
    ldg_words(p, w);
#pragma unroll
    for (int l = 0; l < V; ++l) v[l] = (int)w[l];
  }
  __device__ static C load1(const int* p) {
    u32 w[1];
    ldg_words(p, w);
    return (int)w[0];
  }
  template <int V> __device__ static void store(int* p, const C (&v)[V]) {
    u32 w[V];
#pragma unroll
    for (int l = 0; l < V; ++l) w[l] = (u32)v[l];
    stg_words(p, w);
  }
  __device__ static void store1(int* p, C v) {
    u32 w[1] = {(u32)v};
    stg_words(p, w);
  }
};

template <> struct IO<double> {
  typedef double C;
  template <int V> __device__ static void load(const double* p, C (&v)[V]) {
    u32 w[2 * V];
    ldg_words(p, w);
#pragma unroll
    for (int l = 0; l < V; ++l) v[l] = __hiloint2double((int)w[2 * l + 1], (int)w[2 * l]);
  }
  __device__ static C load1(const double* p) {
    u32 w[2];
    ldg_words(p, w);
    return __hiloint2double((int)w[1], (int)w[0]);
  }
  template <int V> __device__ static void store(double* p, const C (&v)[V]) {
    u32 w[2 * V];
#pragma unroll
    for (int l = 0; l < V; ++l) {
      w[2 * l] = (u32)__double2loint(v[l]);
      w[2 * l + 1] = (u32)__double2hiint(v[l]);
    }
    stg_words(p, w);
  }
  __device__ static void store1(double* p, C v) {
    u32 w[2] = {(u32)__double2loint(v), (u32)__double2hiint(v)};
    stg_words(p, w);
  }
};

template <> struct IO<bf16> {
  typedef float C;
  template <int V> __device__ static void load(const bf16* p, C (&v)[V]) {
    if constexpr (V == 1) {
      v[0] = __uint_as_float(((u32)ldg_u16(p)) << 16);
    } else {
      u32 w[V / 2];
      ldg_words(p, w);
#pragma unroll
      for (int q = 0; q < V / 2; ++q) {
        v[2 * q] = bf16_lo(w[q]);
        v[2 * q + 1] = bf16_hi(w[q]);
      }
    }
  }
  __device__ static C load1(const bf16* p) { return __uint_as_float(((u32)ldg_u16(p)) << 16); }
  // V values from V/2 words already loaded (element 2q in the low half of word q)
  template <int V> __device__ static void convert(const u32 (&w)[V / 2], C (&v)[V]) {
#pragma unroll
    for (int q = 0; q < V / 2; ++q) {
      v[2 * q] = bf16_lo(w[q]);
      v[2 * q + 1] = bf16_hi(w[q]);
    }
  }
  template <int V> __device__ static void store(bf16* p, const C (&v)[V]) {
    if constexpr (V == 1) {
      stg_u16(p, to_bf16(v[0]));
    } else {
      u32 w[V / 2];
#pragma unroll
      for (int q = 0; q < V / 2; ++q) w[q] = pack_bf16x2(v[2 * q], v[2 * q + 1]);
      stg_words(p, w);
    }
  }
  __device__ static void store1(bf16* p, C v) { stg_u16(p, to_bf16(v)); }
};

template <> struct IO<f16> {
  typedef float C;
  template <int V> __device__ static void load(const f16* p, C (&v)[V]) {
    if constexpr (V == 1) {
      v[0] = f16_to_f32(ldg_u16(p));
    } else {
      u32 w[V / 2];
      ldg_words(p, w);
#pragma unroll
      for (int q = 0; q < V / 2; ++q) {
        v[2 * q] = f16_to_f32((u16)(w[q] & 0xffffu));
        v[2 * q + 1] = f16_to_f32((u16)(w[q] >> 16));
      }
    }
  }
  __device__ static C load1(const f16* p) { return f16_to_f32(ldg_u16(p)); }
  template <int V> __device__ static void convert(const u32 (&w)[V / 2], C (&v)[V]) {
#pragma unroll
    for (int q = 0; q < V / 2; ++q) {
      v[2 * q] = f16_to_f32((u16)(w[q] & 0xffffu));
      v[2 * q + 1] = f16_to_f32((u16)(w[q] >> 16));
    }
  }
  template <int V> __device__ static void store(f16* p, const C (&v)[V]) {
    if constexpr (V == 1) {
      stg_u16(p, to_f16(v[0]));
    } else {
      u32 w[V / 2];
#pragma unroll
      for (int q = 0; q < V / 2; ++q) w[q] = pack_f16x2(v[2 * q], v[2 * q + 1]);
      stg_words(p, w);
    }
  }
  __device__ static void store1(f16* p, C v) { stg_u16(p, to_f16(v)); }
};

// ---------------------------------------------------------------------------
// per-node arithmetic in the compute type
// ---------------------------------------------------------------------------
__device__ __forceinline__ float op_add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double op_add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ int op_add(int a, int b) { return (int)((u32)a + (u32)b); }
__device__ __forceinline__ float op_sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double op_sub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ int op_sub(int a, int b) { return (int)((u32)a - (u32)b); }
__device__ __forceinline__ float op_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double op_mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ int op_mul(int a, int b) { return (int)((u32)a * (u32)b); }
__device__ __forceinline__ float op_div(float a, float b, u32&) { return __fdiv_rn(a, b); }
__device__ __forceinline__ double op_div(double a, double b, u32&) { return __ddiv_rn(a, b); }
__device__ __forceinline__ int op_div(int a, int b, u32& err) {
  if (b == 0) {
    err |= 1u;  // COOT_FLAG_INT_DIV_ZERO
    return 0;
  }
  if (a == COOT_INT_MIN && b == -1) return COOT_INT_MIN;  // wraps
  return a / b;                                           // truncates toward zero
}
__device__ __forceinline__ float op_neg(float a) { return -a; }
__device__ __forceinline__ double op_neg(double a) { return -a; }
__device__ __forceinline__ int op_neg(int a) { return (int)(0u - (u32)a); }
__device__ __forceinline__ float op_abs(float a) { return fabsf(a); }
__device__ __forceinline__ double op_abs(double a) { return fabs(a); }
__device__ __forceinline__ int op_abs(int a) { return a < 0 ? (int)(0u - (u32)a) : a; }
__device__ __forceinline__ float op_exp(float a) { return expf(a); }
__device__ __forceinline__ double op_exp(double a) { return exp(a); }
__device__ __forceinline__ float op_log(float a) { return logf(a); }
__device__ __forceinline__ double op_log(double a) { return log(a); }
__device__ __forceinline__ float op_sqrt(float a) { return __fsqrt_rn(a); }
__device__ __forceinline__ double op_sqrt(double a) { return __dsqrt_rn(a); }
__device__ __forceinline__ float op_sign(float a) { return a > 0.f ? 1.f : (a < 0.f ? -1.f : 0.f); }
__device__ __forceinline__ double op_sign(double a) { return a > 0.0 ? 1.0 : (a < 0.0 ? -1.0 : 0.0); }

// scalar of the compute type from its 64-bit pattern
template <class C> __device__ __forceinline__ C scalar_from_bits(u64 b);
template <> __device__ __forceinline__ float scalar_from_bits<float>(u64 b) { return __uint_as_float((u32)b); }
template <> __device__ __forceinline__ double scalar_from_bits<double>(u64 b) { return __longlong_as_double((i64)b); }
template <> __device__ __forceinline__ int scalar_from_bits<int>(u64 b) { return (int)(u32)b; }

// ---------------------------------------------------------------------------
// evaluation context: the loaded leaf values of V consecutive elements, the
// tree's scalars, and a device error word
// ---------------------------------------------------------------------------
template <class C_, int NS, int V> struct Vals {
  typedef C_ C;
  C v[NS > 0 ? NS : 1][V];
};
template <class C, int NK> struct Scal {
  C k[NK > 0 ? NK : 1];
};

// ---------------------------------------------------------------------------
// expression node types (Sec. 3): leaves, eOp and eGlue
// ---------------------------------------------------------------------------
template <int S> struct Leaf {
  template <class X, class K> __device__ __forceinline__ static typename X::C ev(const X& x, const K&, u32&, int l) {
    return x.v[S][l];
  }
  template <class X, class K, class G>
  __device__ __forceinline__ static void bw(const X&, const K&, u32&, int, typename X::C g, G& gs) {
    gs[S] = op_add(gs[S], g);
  }
};

// eOp types: f(a) and the derivative-weighted adjoint d(g) = g * f'(a)
struct eop_neg {
  template <class C, class K> __device__ static C f(C a, const K&, u32&) { return op_neg(a); }
  template <class C, class K> __device__ static C d(C a, C g, const K&, u32&) { return op_neg(g); }
};
struct eop_exp {
  template <class C, class K> __device__ static C f(C a, const K&, u32&) { return op_exp(a); }
  template <class C, class K> __device__ static C d(C a, C g, const K&, u32&) { return op_mul(g, op_exp(a)); }
};
struct eop_log {
  template <class C, class K> __device__ static C f(C a, const K&, u32&) { return op_log(a); }
  template <class C, class K> __device__ static C d(C a, C g, const K&, u32& e) { return op_div(g, a, e); }
};
struct eop_abs {
  template <class C, class K> __device__ static C f(C a, const K&, u32&) { return op_abs(a); }
  template <class C, class K> __device__ static C d(C a, C g, const K&, u32&) { return op_mul(g, op_sign(a)); }
};
struct eop_square {
  template <class C, class K> __device__ static C f(C a, const K&, u32&) { return op_mul(a, a); }
  template <class C, class K> __device__ static C d(C a, C g, const K&, u32&) {
    return op_mul(op_add(g, g), a);
  }
};
struct eop_sqrt {
  template <class C, class K> __device__ static C f(C a, const K&, u32&) { return op_sqrt(a); }
  template <class C, class K> __device__ static C d(C a, C g, const K&, u32& e) {
    C s = op_sqrt(a);
    return op_div(g, op_add(s, s), e);
  }
};
// scalar forms: the scalar is operand K of the tree's scalar table
template <int K_> struct eop_scalar_times {
  template <class C, class K> __device__ static C f(C a, const K& k, u32&) { return op_mul(k.k[K_], a); }
  template <class C, class K> __device__ static C d(C a, C g, const K& k, u32&) { return op_mul(g, k.k[K_]); }
};
template <int K_> struct eop_scalar_plus {
  template <class C, class K> __device__ static C f(C a, const K& k, u32&) { return op_add(a, k.k[K_]); }
  template <class C, class K> __device__ static C d(C a, C g, const K&, u32&) { return g; }
};
template <int K_> struct eop_scalar_minus_pre {  // k - a
  template <class C, class K> __device__ static C f(C a, const K& k, u32&) { return op_sub(k.k[K_], a); }
  template <class C, class K> __device__ static C d(C a, C g, const K&, u32&) { return op_neg(g); }
};
template <int K_> struct eop_scalar_minus_post {  // a - k
  template <class C, class K> __device__ static C f(C a, const K& k, u32&) { return op_sub(a, k.k[K_]); }
  template <class C, class K> __device__ static C d(C a, C g, const K&, u32&) { return g; }
};
template <int K_> struct eop_scalar_div_pre {  // k / a
  template <class C, class K> __device__ static C f(C a, const K& k, u32& e) { return op_div(k.k[K_], a, e); }
  template <class C, class K> __device__ static C d(C a, C g, const K& k, u32& e) {
    // d(k/a)/da = -k / a^2
    return op_neg(op_div(op_mul(g, k.k[K_]), op_mul(a, a), e));
  }
};
template <int K_> struct eop_scalar_div_post {  // a / k
  template <class C, class K> __device__ static C f(C a, const K& k, u32& e) { return op_div(a, k.k[K_], e); }
  template <class C, class K> __device__ static C d(C a, C g, const K& k, u32& e) { return op_div(g, k.k[K_], e); }
};

template <class T1, class Op> struct eOp {
  template <class X, class K> __device__ __forceinline__ static typename X::C ev(const X& x, const K& k, u32& e, int l) {
    return Op::f(T1::ev(x, k, e, l), k, e);
  }
  template <class X, class K, class G>
  __device__ __forceinline__ static void bw(const X& x, const K& k, u32& e, int l, typename X::C g, G& gs) {
    T1::bw(x, k, e, l, Op::d(T1::ev(x, k, e, l), g, k, e), gs);
  }
};

// eGlue types: f(a, b) and the adjoints with respect to a and b
struct eglue_plus {
  template <class C, class K> __device__ static C f(C a, C b, const K&, u32&) { return op_add(a, b); }
  template <class C, class K> __device__ static C da(C, C, C g, const K&, u32&) { return g; }
  template <class C, class K> __device__ static C db(C, C, C g, const K&, u32&) { return g; }
};
struct eglue_minus {
  template <class C, class K> __device__ static C f(C a, C b, const K&, u32&) { return op_sub(a, b); }
  template <class C, class K> __device__ static C da(C, C, C g, const K&, u32&) { return g; }
  template <class C, class K> __device__ static C db(C, C, C g, const K&, u32&) { return op_neg(g); }
};
struct eglue_schur {
  template <class C, class K> __device__ static C f(C a, C b, const K&, u32&) { return op_mul(a, b); }
  template <class C, class K> __device__ static C da(C, C b, C g, const K&, u32&) { return op_mul(g, b); }
  template <class C, class K> __device__ static C db(C a, C, C g, const K&, u32&) { return op_mul(g, a); }
};
struct eglue_div {
  template <class C, class K> __device__ static C f(C a, C b, const K&, u32& e) { return op_div(a, b, e); }
  template <class C, class K> __device__ static C da(C, C b, C g, const K&, u32& e) { return op_div(g, b, e); }
  template <class C, class K> __device__ static C db(C a, C b, C g, const K&, u32& e) {
    // d(a/b)/db = -a / b^2
    return op_neg(op_div(op_mul(g, a), op_mul(b, b), e));
  }
};

template <class T1, class T2, class Op> struct eGlue {
  typedef T1 A;
  typedef T2 B;
  template <class X, class K> __device__ __forceinline__ static typename X::C ev(const X& x, const K& k, u32& e, int l) {
    return Op::f(T1::ev(x, k, e, l), T2::ev(x, k, e, l), k, e);
  }
  template <class X, class K, class G>
  __device__ __forceinline__ static void bw(const X& x, const K& k, u32& e, int l, typename X::C g, G& gs) {
    typename X::C a = T1::ev(x, k, e, l), b = T2::ev(x, k, e, l);
    T1::bw(x, k, e, l, Op::da(a, b, g, k, e), gs);
    T2::bw(x, k, e, l, Op::db(a, b, g, k, e), gs);
  }
};

// ---------------------------------------------------------------------------
// reductions: modes and accumulators
// ---------------------------------------------------------------------------
// reduction modes (RED_*) are defined with the kernel arguments in coot_params.h

// Float-float accumulator (Ogita, Rump and Oishi, "Accurate sum and dot
// product", SIAM J. Sci. Comput. 2005, algorithm Sum2/Dot2): hi is the
// running sum, every TwoSum / TwoProduct error term is added into lo, and
// the result is hi + lo.  Error ~ u|S| + (n u)^2 sum|x| for chain length n.
// COOT_ACCUM_PLAIN / COOT_ACCUM_KAHAN (set per tree, for the accuracy
// comparison) replace the per-term step by a plain FP32 sum or by Kahan's
// compensated summation (lo holds minus Kahan's correction term).
struct AccF {
  float hi, lo;
  __device__ __forceinline__ void init() { hi = 0.f; lo = 0.f; }
  __device__ __forceinline__ void add(float x) {
#if defined(COOT_ACCUM_PLAIN)
    hi = __fadd_rn(hi, x);
#elif defined(COOT_ACCUM_KAHAN)
    float y = __fadd_rn(x, lo);  // lo = -c
    float t = __fadd_rn(hi, y);
    lo = __fsub_rn(y, __fsub_rn(t, hi));
    hi = t;
#else
    float s = __fadd_rn(hi, x);
    float bp = __fsub_rn(s, hi);
    float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(x, bp));
    hi = s;
    lo = __fadd_rn(lo, e);
#endif
  }
  __device__ __forceinline__ void add_prod(float a, float b) {
#if defined(COOT_ACCUM_PLAIN) || defined(COOT_ACCUM_KAHAN)
    add(__fmul_rn(a, b));
#else
    float p = __fmul_rn(a, b);
    float e = __fmaf_rn(a, b, -p);  // exact error of the product
    add(p);
    lo = __fadd_rn(lo, e);
#endif
  }
  __device__ __forceinline__ void merge(const AccF& o) {
    add(o.hi);
    lo = __fadd_rn(lo, o.lo);
  }
  __device__ __forceinline__ AccF shfl_xor(int m) const {
    AccF o;
    o.hi = __shfl_xor_sync(0xffffffffu, hi, m);
    o.lo = __shfl_xor_sync(0xffffffffu, lo, m);
    return o;
  }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// FP64 accumulator: plain double (FP64 runs at 1/64 of the FP32 rate on this
// part; every pass pre-sums its group of loaded values pairwise, so a
// thread's chain has one addition per group).
struct AccD {
  double s;
  __device__ __forceinline__ void init() { s = 0.0; }
  __device__ __forceinline__ void add(double x) { s = __dadd_rn(s, x); }
  __device__ __forceinline__ void add_prod(double a, double b) { s = __dadd_rn(s, __dmul_rn(a, b)); }
  __device__ __forceinline__ void merge(const AccD& o) { s = __dadd_rn(s, o.s); }
  __device__ __forceinline__ AccD shfl_xor(int m) const {
    AccD o;
    o.s = __shfl_xor_sync(0xffffffffu, s, m);
    return o;
  }
  __device__ __forceinline__ double value() const { return s; }
};

// INT32 trees reduce exactly in 64-bit integers (modulo 2^64).
struct AccI {
  u64 s;
  __device__ __forceinline__ void init() { s = 0ull; }
  __device__ __forceinline__ void add(int x) { s += (u64)(i64)x; }
  __device__ __forceinline__ void add_prod(int a, int b) { s += (u64)((i64)a * (i64)b); }
  __device__ __forceinline__ void merge(const AccI& o) { s += o.s; }
  __device__ __forceinline__ AccI shfl_xor(int m) const {
    AccI o;
    o.s = __shfl_xor_sync(0xffffffffu, s, m);
    return o;
  }
  __device__ __forceinline__ i64 ivalue() const { return (i64)s; }
};

template <class C> struct AccOf;
template <> struct AccOf<float> { typedef AccF type; };
template <> struct AccOf<double> { typedef AccD type; };
template <> struct AccOf<int> { typedef AccI type; };

// Extreme value and its position (min, max, index_min, index_max).  The
// empty state is (the identity of the order: +inf for min, -inf for max,
// INT_MAX / INT_MIN for integers; position "none" = 2^63-1), so that
//   take y  <=>  y beats v, or y == v and y comes first
// needs no separate test for NaN (every comparison with NaN is false, so NaN
// is never taken) nor for the empty state (an empty partner ties on v and
// loses on position).  Equal values keep the smallest position, which makes
// the result independent of the order of visits and merges.
constexpr i64 POS_NONE = 0x7fffffffffffffffll;
template <class C> struct Lim;
template <> struct Lim<float> {
  __device__ static float hi() { return __int_as_float(0x7f800000); }
  __device__ static float lo() { return __int_as_float((int)0xff800000u); }
};
template <> struct Lim<double> {
  __device__ static double hi() { return __longlong_as_double(0x7ff0000000000000ll); }
  __device__ static double lo() { return __longlong_as_double((i64)0xfff0000000000000ull); }
};
template <> struct Lim<int> {
  __device__ static int hi() { return 0x7fffffff; }
  __device__ static int lo() { return (int)0x80000000u; }
};
template <class C, bool MAX> struct AccExt {
  C v;
  i64 pos;
  __device__ __forceinline__ void init() {
    v = MAX ? Lim<C>::lo() : Lim<C>::hi();
    pos = POS_NONE;
  }
  __device__ __forceinline__ void add_at(C y, i64 q) {
    const bool take = (MAX ? (y > v) : (y < v)) || (y == v && q < pos);
    v = take ? y : v;
    pos = take ? q : pos;
  }
  __device__ __forceinline__ void merge(const AccExt& o) { add_at(o.v, o.pos); }
  __device__ __forceinline__ AccExt shfl_xor(int m) const {
    AccExt o;
    o.v = __shfl_xor_sync(0xffffffffu, v, m);
    o.pos = __shfl_xor_sync(0xffffffffu, pos, m);
    return o;
  }
};

// Products keep their binary exponent apart from the significand, so that no
// partial product overflows or underflows: every factor is split as
// x = m 2^e with |m| in [0.5, 1) (IEEE 754 fields; subnormals are scaled by
// 2^64 first), the running significand is renormalised to [0.5, 1) after
// each step and the exponents are summed in 64-bit integers.  Zeros,
// infinities and NaN pass through the significand unchanged (exponent 0), so
// they propagate as in an ordinary product.
__device__ __forceinline__ float split_exp(float x, i64& e) {
  u32 b = __float_as_uint(x);
  int be = (int)((b >> 23) & 0xffu);
  i64 adj = 0;
  if (be == 0 && (b & 0x7fffffffu) != 0u) {  // subnormal: scale by 2^64
    x = __fmul_rn(x, __uint_as_float(0x5f800000u));
    b = __float_as_uint(x);
    be = (int)((b >> 23) & 0xffu);
    adj = -64;
  }
  if (be == 0 || be == 255) return x;  // zero, inf, NaN
  e += (i64)(be - 126) + adj;
  return __uint_as_float((b & 0x807fffffu) | (126u << 23));
}
__device__ __forceinline__ double split_exp(double x, i64& e) {
  u64 b = (u64)__double_as_longlong(x);
  int be = (int)((b >> 52) & 0x7ffull);
  i64 adj = 0;
  if (be == 0 && (b & 0x7fffffffffffffffull) != 0ull) {
    x = __dmul_rn(x, __longlong_as_double(0x43f0000000000000ll));  // 2^64
    b = (u64)__double_as_longlong(x);
    be = (int)((b >> 52) & 0x7ffull);
    adj = -64;
  }
  if (be == 0 || be == 2047) return x;
  e += (i64)(be - 1022) + adj;
  return __longlong_as_double((i64)((b & 0x800fffffffffffffull) | (1022ull << 52)));
}
// v 2^e in double, saturating to 0 / inf outside the double range
__device__ __forceinline__ double scale2(double v, i64 e) {
  if (v == 0.0 || !(v - v == 0.0)) return v;
  if (e > 2100) e = 2100;
  if (e < -2200) e = -2200;
  return scalbn(v, (int)e);
}

// FP32: float-float significand (TwoProduct through fma: hi*m exactly equals
// p + err), relative error ~ (n u)^2 + u.  The running significand is kept
// in [2^-32, 2^32] and a factor in that range is used as it is (their
// product stays inside [2^-64, 2^64], far from overflow and from the
// subnormal range, also for lo); only other factors are split, and hi is
// renormalised only when it leaves the range.
struct AccProdF {
  float hi, lo;
  i64 e;
  __device__ __forceinline__ void init() { hi = 1.f; lo = 0.f; e = 0; }
  __device__ static __forceinline__ bool in_range(float a) {
    const float m = fabsf(a);
    return m >= 2.3283064365386963e-10f && m <= 4294967296.0f;  // 2^-32, 2^32
  }
  __device__ __forceinline__ void renorm() {
    i64 d = 0;
    float h = split_exp(hi, d);
    if (d != 0) {
      lo = __fmul_rn(lo, __uint_as_float((u32)(127 - d) << 23));  // 2^-d, |d| <= 65
      hi = h;
      e += d;
    }
  }
  __device__ __forceinline__ void mul(float x) {
    float m = x;
    if (!in_range(x)) m = split_exp(x, e);  // also zero, subnormal, inf, NaN
    float p = __fmul_rn(hi, m);
    float err = __fmaf_rn(hi, m, -p);
    lo = __fmaf_rn(lo, m, err);
    hi = p;
    if (!in_range(hi)) renorm();
  }
  __device__ __forceinline__ void merge(const AccProdF& o) {
    float p = __fmul_rn(hi, o.hi);
    float err = __fmaf_rn(hi, o.hi, -p);
    lo = __fmaf_rn(hi, o.lo, __fmaf_rn(lo, o.hi, err));
    hi = p;
    e += o.e;
    renorm();
  }
  __device__ __forceinline__ AccProdF shfl_xor(int m) const {
    AccProdF o;
    o.hi = __shfl_xor_sync(0xffffffffu, hi, m);
    o.lo = __shfl_xor_sync(0xffffffffu, lo, m);
    o.e = __shfl_xor_sync(0xffffffffu, e, m);
    return o;
  }
  __device__ __forceinline__ double value() const {
    if (hi == 0.f || !(hi - hi == 0.f)) return (double)hi;
    return scale2((double)hi + (double)lo, e);
  }
};
// FP64: plain double significand (relative error ~ n u for a chain of n).
// Same scheme with the range [2^-300, 2^300], tested on the biased exponent
// in integer arithmetic (FP64 compares share the slow FP64 pipe).
struct AccProdD {
  double hi;
  i64 e;
  __device__ __forceinline__ void init() { hi = 1.0; e = 0; }
  __device__ static __forceinline__ bool in_range(double a) {
    const u32 be = ((u32)__double2hiint(a) >> 20) & 0x7ffu;
    return be - (1023u - 300u) <= 600u;
  }
  __device__ __forceinline__ void renorm() {
    i64 d = 0;
    double h = split_exp(hi, d);
    hi = h;
    e += d;
  }
  __device__ __forceinline__ void mul(double x) {
    double m = x;
    if (!in_range(x)) m = split_exp(x, e);
    hi = __dmul_rn(hi, m);
    if (!in_range(hi)) renorm();
  }
  __device__ __forceinline__ void merge(const AccProdD& o) {
    hi = __dmul_rn(hi, o.hi);
    e += o.e;
    renorm();
  }
  __device__ __forceinline__ AccProdD shfl_xor(int m) const {
    AccProdD o;
    o.hi = __shfl_xor_sync(0xffffffffu, hi, m);
    o.e = __shfl_xor_sync(0xffffffffu, e, m);
    return o;
  }
  __device__ __forceinline__ double value() const { return scale2(hi, e); }
};
// INT32: exact product modulo 2^64
struct AccProdI {
  u64 s;
  __device__ __forceinline__ void init() { s = 1ull; }
  __device__ __forceinline__ void mul(int x) { s *= (u64)(i64)x; }
  __device__ __forceinline__ void merge(const AccProdI& o) { s *= o.s; }
  __device__ __forceinline__ AccProdI shfl_xor(int m) const {
    AccProdI o;
    o.s = __shfl_xor_sync(0xffffffffu, s, m);
    return o;
  }
  __device__ __forceinline__ i64 ivalue() const { return (i64)s; }
};
template <class C> struct ProdOf;
template <> struct ProdOf<float> { typedef AccProdF type; };
template <> struct ProdOf<double> { typedef AccProdD type; };
template <> struct ProdOf<int> { typedef AccProdI type; };

// the accumulator of a reduction mode
template <class C, int RED> struct AccSel { typedef typename AccOf<C>::type type; };
template <class C> struct AccSel<C, RED_MIN> { typedef AccExt<C, false> type; };
template <class C> struct AccSel<C, RED_IMIN> { typedef AccExt<C, false> type; };
template <class C> struct AccSel<C, RED_MAX> { typedef AccExt<C, true> type; };
template <class C> struct AccSel<C, RED_IMAX> { typedef AccExt<C, true> type; };
template <class C> struct AccSel<C, RED_PROD> { typedef typename ProdOf<C>::type type; };

// Centred sum of squares for the second pass of var.  The mean arrives as a
// double m; FP32 data keeps it as the float pair (mh, ml) = m and forms
// d = (x - mh) - ml: each subtraction's rounding error is at most u |d| (the
// first result is d + ml, the second d), so d carries a relative error of at
// most 2u for any ratio of mean to spread, and the low part ml removes the
// bias a rounded mean would add to every term.  The d*d are all positive, so
// their rounding errors cannot cancel into a large relative error; they are
// accumulated in float-float.  FP64 data uses plain FP64.
struct CsqF {
  float mh, ml;
  __device__ __forceinline__ void set_mean(double m) {
    mh = __double2float_rn(m);
    ml = __double2float_rn(m - (double)mh);
  }
  __device__ __forceinline__ float centred(float x) const { return __fsub_rn(__fsub_rn(x, mh), ml); }
};
struct CsqD {
  double m;
  __device__ __forceinline__ void set_mean(double mm) { m = mm; }
  __device__ __forceinline__ double centred(double x) const { return __dsub_rn(x, m); }
};
template <class C> struct CsqOf;
template <> struct CsqOf<float> { typedef CsqF type; };
template <> struct CsqOf<double> { typedef CsqD type; };
template <> struct CsqOf<int> { typedef CsqD type; };  // never instantiated for int trees

// warp and block reduction in a fixed order (deterministic run to run)
template <class A> __device__ __forceinline__ A warp_reduce(A a) {
#pragma unroll
  for (int m = 16; m >= 1; m >>= 1) a.merge(a.shfl_xor(m));
  return a;
}

template <class A> __device__ __forceinline__ A block_reduce(A a, A* smem) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
  a = warp_reduce(a);
  __syncthreads();
  if (lane == 0) smem[warp] = a;
  __syncthreads();
  if (warp == 0) {
    A b;
    b.init();
    if (lane < nw) b = smem[lane];
    b = warp_reduce(b);
    a = b;
  }
  return a;  // valid in thread 0
}

template <class A> __device__ __forceinline__ A load_volatile(const A* p) {
  A r;
  const volatile unsigned int* src = (const volatile unsigned int*)p;
  unsigned int* dst = (unsigned int*)&r;
#pragma unroll
  for (int i = 0; i < (int)(sizeof(A) / 4); ++i) dst[i] = src[i];
  return r;
}

}  // namespace coot
