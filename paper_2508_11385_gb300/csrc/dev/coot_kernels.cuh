// coot_kernels.cuh -- kernel bodies instantiated per expression tree.
//
// Families (one generated __global__ wrapper per instantiation):
//   str   element-wise map over a column-major 2-D range without transposed
//         reads (a contiguous tree is walked as one long column), with an
//         optional full reduction; 128-bit vector loads/stores when every
//         read and the output are 16-byte aligned along columns.
//   col   the same map with a per-column reduction (sum/mean along dim 0):
//         a group of warps per column.
//   row   the same map with a per-row reduction (dim 1): a thread owns V
//         consecutive rows and walks a range of columns; column ranges are
//         combined by the last block of each row block.
//   tile  any tree with transposed reads: 32x32 output tiles, transposed
//         reads staged through a padded shared-memory tile so that both the
//         read and the write are coalesced; full, dim-0 and dim-1 reductions.
//   adj   fused adjoint of a scalar loss sum(tree): forward values are
//         recomputed per element and the reverse sweep writes every leaf's
//         gradient.
//   batch persistent kernel over many problems pulling chunks of 32x32 tiles
//         from a queue, with a per-problem reduction.
// Cross-block combines use a ticket counter: the block that arrives last
// combines the partials in a fixed order and resets the counter.  Nothing
// ever waits on another block.
#pragma once
#include "coot_params.h"
#include "coot_dev.cuh"

namespace coot {

// ld.global.cg: read a value another block wrote (at L2, not L1)
template <class A> __device__ __forceinline__ A load_cg(const A* p) {
  A r;
  const unsigned int* src = (const unsigned int*)p;
  unsigned int* dst = (unsigned int*)&r;
#pragma unroll
  for (int i = 0; i < (int)(sizeof(A) / 4); ++i) asm volatile("ld.global.cg.u32 %0, [%1];" : "=r"(dst[i]) : "l"(src + i));
  return r;
}

template <class S> __device__ __forceinline__ const S* at(const void* base, long long i, long long j, long long ld) {
  return (const S*)base + (i + j * ld);
}
template <class S> __device__ __forceinline__ S* at_out(void* base, long long i, long long j, long long ld) {
  return (S*)base + (i + j * ld);
}

// ---------------------------------------------------------------------------
// per-element contribution of the root to the reduction
// ---------------------------------------------------------------------------
// pos: the element's position in its reduction (column-major linear index for
// a full reduction, row index along dim 0, column index along dim 1); only
// index_min / index_max read it (and min / max, to keep the first of equal
// values), everywhere else the expression is dead code.
template <class T, int RED, class X, class K, class A, class Q>
__device__ __forceinline__ typename X::C eval_elem(const X& x, const K& k, u32& err, int l, A& acc, const Q& csq,
                                                   long long pos) {
  typedef typename X::C C;
  if constexpr (red_extreme(RED)) {
    C y = T::ev(x, k, err, l);
    acc.add_at(y, pos);
    return y;
  } else if constexpr (RED == RED_PROD) {
    C y = T::ev(x, k, err, l);
    acc.mul(y);
    return y;
  } else if constexpr (RED == RED_DOT) {
    C a = T::A::ev(x, k, err, l), b = T::B::ev(x, k, err, l);
    acc.add_prod(a, b);
    return op_mul(a, b);
  } else {
    C y = T::ev(x, k, err, l);
    if constexpr (RED == RED_SUM || RED == RED_MEAN1) acc.add(y);
    if constexpr (RED == RED_SSQ) acc.add_prod(y, y);
    if constexpr (RED == RED_CSQ) {
      C d = csq.centred(y);
      acc.add(op_mul(d, d));
    }
    return y;
  }
}

// The element's value y and, in c, its term of the reduction, for the
// pairwise path of 16-bit storage: products and squares of two 16-bit values
// are exact in FP32 (at most 22 significant bits), and sums of two such terms
// are exact unless their exponents differ by more than 15, so the V terms of
// one vector load are summed pairwise in FP32 before a single float-float
// addition.
template <class T, int RED, class X, class K, class Q>
__device__ __forceinline__ typename X::C eval_term(const X& x, const K& k, u32& err, int l, const Q& csq,
                                                   typename X::C& c) {
  typedef typename X::C C;
  if constexpr (RED == RED_DOT) {
    C a = T::A::ev(x, k, err, l), b = T::B::ev(x, k, err, l);
    c = op_mul(a, b);
    return c;
  } else {
    C y = T::ev(x, k, err, l);
    if constexpr (RED == RED_SSQ) c = op_mul(y, y);
    else if constexpr (RED == RED_CSQ) {
      C d = csq.centred(y);
      c = op_mul(d, d);
    } else
      c = y;
    return y;
  }
}

// the final value written for one reduction output
template <class C, int RED, class A>
__device__ __forceinline__ void write_result(const Params& p, const A& a, long long idx, double div) {
  typedef typename rtype<C>::type R;
  const double qnan = __longlong_as_double(0x7ff8000000000000ll);
  if constexpr (RED == RED_IMIN || RED == RED_IMAX) {
    // positions are int64 for every element type; -1: no element (or all NaN)
    ((long long*)p.red_out)[idx] = (a.pos == POS_NONE) ? -1ll : (long long)a.pos;
  } else if constexpr (RED == RED_MIN || RED == RED_MAX) {
    if constexpr (is_int_c<C>::value)
      ((long long*)p.red_out)[idx] = (a.pos == POS_NONE) ? 0ll : (long long)a.v;
    else
      ((R*)p.red_out)[idx] = (a.pos == POS_NONE) ? (R)qnan : (R)a.v;
  } else if constexpr (is_int_c<C>::value) {
    // integer trees: exact int64 sums and products (sum / dot / prod)
    ((long long*)p.red_out)[idx] = a.ivalue();
  } else {
    if constexpr (RED == RED_SUM || RED == RED_DOT) {
      ((R*)p.red_out)[idx] = (R)(a.value() / div);
    } else if constexpr (RED == RED_PROD) {
      ((R*)p.red_out)[idx] = (R)a.value();
    } else if constexpr (RED == RED_SSQ) {
      ((R*)p.red_out)[idx] = (R)sqrt(a.value());
    } else if constexpr (RED == RED_MEAN1) {
      p.mu[idx] = a.value() / (double)p.count;  // count: elements per output
    } else if constexpr (RED == RED_CSQ) {
      double v;
      if (p.count == 0)
        v = qnan;  // no elements
      else if (p.count == 1)
        v = 0.0;
      else
        v = a.value() / p.den;
      if (p.flags & PF_SQRT) v = sqrt(v);
      ((R*)p.red_out)[idx] = (R)v;
    }
  }
}

// block-level partial -> ticket -> last block combines all partials in order
template <class C, int RED, class A> __device__ __forceinline__ void finish_full(const Params& p, A acc, A* smem) {
  __shared__ int am_last;
  acc = block_reduce(acc, smem);
  if (threadIdx.x == 0) {
    ((A*)p.partials)[blockIdx.x] = acc;
    __threadfence();
    unsigned int t = atomicAdd(p.tickets, 1u);
    am_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (am_last) {
    __threadfence();
    A a;
    a.init();
    for (unsigned int b = threadIdx.x; b < gridDim.x; b += blockDim.x) a.merge(load_cg(&((const A*)p.partials)[b]));
    a = block_reduce(a, smem);
    if (threadIdx.x == 0) {
      write_result<C, RED>(p, a, 0, p.div);
      *p.tickets = 0u;  // ready for the next launch
    }
  }
}

// ---------------------------------------------------------------------------
// str: map (+ full reduction) over n_rows x n_cols, no transposed reads
// ---------------------------------------------------------------------------
template <class T, class S, int NS, int NK, int RED, int V, int U, bool OUT>
__device__ __forceinline__ void str_kernel(const Params& p) {
  typedef typename ctype<S>::type C;
  typedef typename AccSel<C, RED>::type A;
  __shared__ A smem[32];
  Scal<C, NK> k;
#pragma unroll
  for (int q = 0; q < NK; ++q) k.k[q] = scalar_from_bits<C>(p.k[q]);
  typename CsqOf<C>::type csq;
  if constexpr (RED == RED_CSQ) csq.set_mean(*p.mu);
  u32 err = 0;
  // one accumulator per vector lane: V independent addition chains
  A accs[V];
#pragma unroll
  for (int l = 0; l < V; ++l) accs[l].init();
  const long long nr = p.n_rows, nc = p.n_cols, cpc = p.units_per_col;
  const long long units = cpc * nc;
  const long long step = (long long)blockDim.x * V;
  const long long CH = step * U;
  for (long long u = blockIdx.x; u < units; u += gridDim.x) {
    const long long j = (nc == 1) ? 0 : u / cpc;
    const long long i0 = (u - j * cpc) * CH + (long long)threadIdx.x * V;
    Vals<C, NS, V> x[U];
    bool full[U];
#pragma unroll
    for (int g = 0; g < U; ++g) {
      const long long i = i0 + g * step;
      full[g] = (i + V <= nr);
      if (full[g]) {
#pragma unroll
        for (int s = 0; s < NS; ++s) IO<S>::template load<V>(at<S>(p.src[s], i, j, p.ld[s]), x[g].v[s]);
      } else {
#pragma unroll
        for (int s = 0; s < NS; ++s)
#pragma unroll
          for (int l = 0; l < V; ++l) x[g].v[s][l] = (i + l < nr) ? IO<S>::load1(at<S>(p.src[s], i + l, j, p.ld[s])) : C(0);
      }
    }
#pragma unroll
    for (int g = 0; g < U; ++g) {
      const long long i = i0 + g * step;
      if (full[g]) {
        C y[V];
        if constexpr (sizeof(S) == 2 && red_additive(RED)) {
          // 16-bit storage: pairwise sum of the vector's terms, then one
          // float-float addition (spread over the accumulators by group)
          C c[V];
#pragma unroll
          for (int l = 0; l < V; ++l) y[l] = eval_term<T, RED>(x[g], k, err, l, csq, c[l]);
#pragma unroll
          for (int w = V / 2; w >= 1; w /= 2)
#pragma unroll
            for (int l = 0; l < w; ++l) c[l] = op_add(c[l], c[l + w]);
          accs[g % V].add(c[0]);
        } else {
#pragma unroll
          for (int l = 0; l < V; ++l) y[l] = eval_elem<T, RED>(x[g], k, err, l, accs[l], csq, i + l + j * nr);
        }
        if constexpr (OUT) IO<S>::template store<V>(at_out<S>(p.out, i, j, p.out_ld), y);
      } else {
#pragma unroll
        for (int l = 0; l < V; ++l)
          if (i + l < nr) {
            C y = eval_elem<T, RED>(x[g], k, err, l, accs[l], csq, i + l + j * nr);
            if constexpr (OUT) IO<S>::store1(at_out<S>(p.out, i + l, j, p.out_ld), y);
          }
      }
    }
  }
  if (err) atomicOr(p.err_flag, err);
  if constexpr (RED != RED_NONE) {
#pragma unroll
    for (int l = 1; l < V; ++l) accs[0].merge(accs[l]);
    finish_full<C, RED>(p, accs[0], smem);
  }
}

// ---------------------------------------------------------------------------
// col: map + per-column reduction (dim 0).  A group of G warps (G =
// p.n_splits, a divisor of the warps per block) owns one column at a time and
// splits its rows; the group's warp results are combined in shared memory in
// warp order.  Every block runs the same number of column steps, so the
// barriers are uniform.
// ---------------------------------------------------------------------------
template <class T, class S, int NS, int NK, int RED, int V, int U, bool OUT>
__device__ __forceinline__ void col_kernel(const Params& p) {
  typedef typename ctype<S>::type C;
  typedef typename AccSel<C, RED>::type A;
  __shared__ A wsum[32];
  Scal<C, NK> k;
#pragma unroll
  for (int q = 0; q < NK; ++q) k.k[q] = scalar_from_bits<C>(p.k[q]);
  typename CsqOf<C>::type csq;
  u32 err = 0;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long wpb = blockDim.x >> 5;
  const long long G = p.n_splits;  // warps per column
  const long long gpb = wpb / G;   // columns per block step
  const long long gi = warp / G, wm = warp % G;
  const long long nr = p.n_rows, nc = p.n_cols;
  const long long step = 32LL * V;
  for (long long base = (long long)blockIdx.x * gpb; base < nc; base += (long long)gridDim.x * gpb) {
    const long long j = base + gi;
    A acc;
    acc.init();
    if constexpr (RED == RED_CSQ) csq.set_mean(p.mu[j < nc ? j : 0]);
    for (long long i0 = (wm * 32 + lane) * V; j < nc && i0 < nr; i0 += G * step * U) {
      Vals<C, NS, V> x[U];
      bool full[U];
#pragma unroll
      for (int g = 0; g < U; ++g) {
        const long long i = i0 + g * G * step;
        full[g] = (i + V <= nr);
        if (full[g]) {
#pragma unroll
          for (int s = 0; s < NS; ++s) IO<S>::template load<V>(at<S>(p.src[s], i, j, p.ld[s]), x[g].v[s]);
        } else {
#pragma unroll
          for (int s = 0; s < NS; ++s)
#pragma unroll
            for (int l = 0; l < V; ++l)
              x[g].v[s][l] = (i + l < nr) ? IO<S>::load1(at<S>(p.src[s], i + l, j, p.ld[s])) : C(0);
        }
      }
#pragma unroll
      for (int g = 0; g < U; ++g) {
        const long long i = i0 + g * G * step;
        if (full[g]) {
          C y[V];
#pragma unroll
          for (int l = 0; l < V; ++l) y[l] = eval_elem<T, RED>(x[g], k, err, l, acc, csq, i + l);
          if constexpr (OUT) IO<S>::template store<V>(at_out<S>(p.out, i, j, p.out_ld), y);
        } else {
#pragma unroll
          for (int l = 0; l < V; ++l)
            if (i + l < nr) {
              C y = eval_elem<T, RED>(x[g], k, err, l, acc, csq, i + l);
              if constexpr (OUT) IO<S>::store1(at_out<S>(p.out, i + l, j, p.out_ld), y);
            }
        }
      }
    }
    acc = warp_reduce(acc);
    if (G == 1) {
      if (lane == 0 && j < nc) write_result<C, RED>(p, acc, j, p.div);
    } else {
      if (lane == 0) wsum[warp] = acc;
      __syncthreads();
      if (wm == 0 && lane == 0 && j < nc) {
        A a = wsum[gi * G];
        for (long long w = 1; w < G; ++w) a.merge(wsum[gi * G + w]);
        write_result<C, RED>(p, a, j, p.div);
      }
      __syncthreads();
    }
  }
  if (err) atomicOr(p.err_flag, err);
}

// ---------------------------------------------------------------------------
// row: map + per-row reduction (dim 1)
//   block b -> row block rb = b % n_row_blocks, column split sp = b / n_row_blocks
// ---------------------------------------------------------------------------
template <class T, class S, int NS, int NK, int RED, int V, int U, bool OUT>
__device__ __forceinline__ void row_kernel(const Params& p) {
  typedef typename ctype<S>::type C;
  typedef typename AccSel<C, RED>::type A;
  __shared__ int am_last;
  Scal<C, NK> k;
#pragma unroll
  for (int q = 0; q < NK; ++q) k.k[q] = scalar_from_bits<C>(p.k[q]);
  u32 err = 0;
  const long long nr = p.n_rows, nc = p.n_cols;
  const long long nrb = p.n_row_blocks, nsp = p.n_splits, cps = p.units_per_col;
  const long long rb = blockIdx.x % nrb, sp = blockIdx.x / nrb;
  const long long i = (rb * blockDim.x + threadIdx.x) * V;
  const long long j0 = sp * cps;
  const long long j1 = (j0 + cps < nc) ? j0 + cps : nc;
  const bool fullv = (i + V <= nr);
  A acc[V];
  typename CsqOf<C>::type csq[V];  // var along dim 1: one mean per row
#pragma unroll
  for (int l = 0; l < V; ++l) {
    acc[l].init();
    if constexpr (RED == RED_CSQ) csq[l].set_mean(i + l < nr ? p.mu[i + l] : 0.0);
  }
  if (i < nr) {
    for (long long jb = j0; jb < j1; jb += U) {
      Vals<C, NS, V> x[U];
#pragma unroll
      for (int g = 0; g < U; ++g) {
        const long long j = jb + g;
        if (j < j1) {
          if (fullv) {
#pragma unroll
            for (int s = 0; s < NS; ++s) IO<S>::template load<V>(at<S>(p.src[s], i, j, p.ld[s]), x[g].v[s]);
          } else {
#pragma unroll
            for (int s = 0; s < NS; ++s)
#pragma unroll
              for (int l = 0; l < V; ++l)
                x[g].v[s][l] = (i + l < nr) ? IO<S>::load1(at<S>(p.src[s], i + l, j, p.ld[s])) : C(0);
          }
        }
      }
#pragma unroll
      for (int g = 0; g < U; ++g) {
        const long long j = jb + g;
        if (j < j1) {
          if (fullv) {
            C y[V];
#pragma unroll
            for (int l = 0; l < V; ++l) y[l] = eval_elem<T, RED>(x[g], k, err, l, acc[l], csq[l], j);
            if constexpr (OUT) IO<S>::template store<V>(at_out<S>(p.out, i, j, p.out_ld), y);
          } else {
#pragma unroll
            for (int l = 0; l < V; ++l)
              if (i + l < nr) {
                C y = eval_elem<T, RED>(x[g], k, err, l, acc[l], csq[l], j);
                if constexpr (OUT) IO<S>::store1(at_out<S>(p.out, i + l, j, p.out_ld), y);
              }
          }
        }
      }
    }
  }
  if (err) atomicOr(p.err_flag, err);
  if (nsp == 1) {
#pragma unroll
    for (int l = 0; l < V; ++l)
      if (i + l < nr) write_result<C, RED>(p, acc[l], i + l, p.div);
    return;
  }
#pragma unroll
  for (int l = 0; l < V; ++l)
    if (i + l < nr) ((A*)p.partials)[sp * nr + i + l] = acc[l];
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned int t = atomicAdd(&p.tickets[rb], 1u);
    am_last = (t == (unsigned int)(nsp - 1));
  }
  __syncthreads();
  if (am_last) {
    __threadfence();
#pragma unroll
    for (int l = 0; l < V; ++l)
      if (i + l < nr) {
        A a;
        a.init();
        for (long long s = 0; s < nsp; ++s) a.merge(load_cg(&((const A*)p.partials)[s * nr + i + l]));
        write_result<C, RED>(p, a, i + l, p.div);
      }
    if (threadIdx.x == 0) p.tickets[rb] = 0u;
  }
}

// ---------------------------------------------------------------------------
// tile: any tree with transposed reads; TRMASK marks the transposed slots.
//   32x32 output tile, 256 threads as 32 (rows) x 8 (column phases); each
//   thread evaluates rows i = 32 ti + tx of columns j = 32 tj + ty + 8 q.
//   A transposed slot reads view(j, i): its 32x32 source block is read with
//   consecutive threads on consecutive source rows and parked in shared
//   memory with one column of padding, then read back transposed.
//   DIM: -1 full reduction, 0 per column, 1 per row.
// ---------------------------------------------------------------------------
constexpr int TILE = 32;
constexpr int TILE_PH = 8;  // blockDim.x == TILE * TILE_PH
constexpr int TILE_Q = TILE / TILE_PH;

template <int M> struct popc { static constexpr int value = (M & 1) + popc<(M >> 1)>::value; };
template <> struct popc<0> { static constexpr int value = 0; };

template <class T, class S, int NS, int NK, int RED, int DIM, int TRMASK, bool OUT>
__device__ __forceinline__ void tile_kernel(const Params& p) {
  typedef typename ctype<S>::type C;
  typedef typename AccSel<C, RED>::type A;
  constexpr int NTR = popc<TRMASK>::value;
  __shared__ C stage[NTR > 0 ? NTR : 1][TILE][TILE + 1];
  __shared__ A smem[32];
  __shared__ A rsum[TILE_PH][TILE];
  __shared__ int am_last;
  Scal<C, NK> k;
#pragma unroll
  for (int q = 0; q < NK; ++q) k.k[q] = scalar_from_bits<C>(p.k[q]);
  typename CsqOf<C>::type csq;
  if constexpr (RED == RED_CSQ && DIM == -1) csq.set_mean(*p.mu);
  u32 err = 0;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const long long nr = p.n_rows, nc = p.n_cols;
  const long long ntr = (nr + TILE - 1) / TILE, ntc = (nc + TILE - 1) / TILE;
  const long long tiles = ntr * ntc;
  A acc;
  acc.init();
  for (long long t = blockIdx.x; t < tiles; t += gridDim.x) {
    const long long ti = t % ntr, tj = t / ntr;
    const long long i = ti * TILE + tx;
    Vals<C, NS, TILE_Q> x;
    // direct reads first: they stay in flight while transposed blocks are staged
#pragma unroll
    for (int w = 0; w < TILE_Q; ++w) {
      const long long j = tj * TILE + ty + TILE_PH * w;
      const bool ok = (i < nr && j < nc);
#pragma unroll
      for (int s = 0; s < NS; ++s)
        if (!((TRMASK >> s) & 1)) x.v[s][w] = ok ? IO<S>::load1(at<S>(p.src[s], i, j, p.ld[s])) : C(0);
    }
    if constexpr (NTR > 0) {
      __syncthreads();  // the previous tile's shared reads are done
      int q = 0;
#pragma unroll
      for (int s = 0; s < NS; ++s)
        if ((TRMASK >> s) & 1) {
          const long long vr = tj * TILE + tx;  // view row  = output column
#pragma unroll
          for (int w = 0; w < TILE_Q; ++w) {
            const long long vc = ti * TILE + ty + TILE_PH * w;  // view column = output row
            stage[q][ty + TILE_PH * w][tx] = (vr < nc && vc < nr) ? IO<S>::load1(at<S>(p.src[s], vr, vc, p.ld[s])) : C(0);
          }
          ++q;
        }
      __syncthreads();
      q = 0;
#pragma unroll
      for (int s = 0; s < NS; ++s)
        if ((TRMASK >> s) & 1) {
#pragma unroll
          for (int w = 0; w < TILE_Q; ++w) x.v[s][w] = stage[q][tx][ty + TILE_PH * w];
          ++q;
        }
    }
    A racc;  // per-row partial over this tile's columns (DIM 1)
    racc.init();
#pragma unroll
    for (int w = 0; w < TILE_Q; ++w) {
      const long long j = tj * TILE + ty + TILE_PH * w;
      const bool ok = (i < nr && j < nc);
      if constexpr (DIM == 0) {
        A cacc;
        cacc.init();
        if (ok) {
          if constexpr (RED == RED_CSQ) csq.set_mean(p.mu[j]);
          C y = eval_elem<T, RED>(x, k, err, w, cacc, csq, i);
          if constexpr (OUT) IO<S>::store1(at_out<S>(p.out, i, j, p.out_ld), y);
        }
        cacc = warp_reduce(cacc);  // the 32 rows of column j
        if (tx == 0 && j < nc) ((A*)p.partials)[ti * nc + j] = cacc;
      } else if constexpr (DIM == 1) {
        if (ok) {
          if constexpr (RED == RED_CSQ) csq.set_mean(p.mu[i]);
          C y = eval_elem<T, RED>(x, k, err, w, racc, csq, j);
          if constexpr (OUT) IO<S>::store1(at_out<S>(p.out, i, j, p.out_ld), y);
        }
      } else {
        if (ok) {
          C y = eval_elem<T, RED>(x, k, err, w, acc, csq, i + j * nr);
          if constexpr (OUT) IO<S>::store1(at_out<S>(p.out, i, j, p.out_ld), y);
        }
      }
    }
    if constexpr (DIM == 1) {
      rsum[ty][tx] = racc;
      __syncthreads();
      if (ty == 0) {
        A a = rsum[0][tx];
        for (int r = 1; r < TILE_PH; ++r) a.merge(rsum[r][tx]);
        if (i < nr) ((A*)p.partials)[tj * nr + i] = a;
      }
    }
    if constexpr (DIM == 0 || DIM == 1) {
      // last tile of a column strip (DIM 0) / row strip (DIM 1) combines
      __threadfence();
      __syncthreads();
      const long long strip = (DIM == 0) ? tj : ti;
      const long long need = (DIM == 0) ? ntr : ntc;
      if (threadIdx.x == 0) {
        unsigned int tk = atomicAdd(&p.tickets[strip], 1u);
        am_last = (tk == (unsigned int)(need - 1));
      }
      __syncthreads();
      if (am_last) {
        __threadfence();
        // thread (tx, ty): output o = 32 strip + tx, partials ty, ty+8, ...
        const long long o = strip * TILE + tx;
        const long long no = (DIM == 0) ? nc : nr;
        A a;
        a.init();
        if (o < no)
          for (long long s = ty; s < need; s += TILE_PH) a.merge(load_cg(&((const A*)p.partials)[s * no + o]));
        rsum[ty][tx] = a;
        __syncthreads();
        if (ty == 0 && o < no) {
          A b = rsum[0][tx];
          for (int r = 1; r < TILE_PH; ++r) b.merge(rsum[r][tx]);
          write_result<C, RED>(p, b, o, p.div);
        }
        if (threadIdx.x == 0) p.tickets[strip] = 0u;
      }
      __syncthreads();
    }
  }
  if (err) atomicOr(p.err_flag, err);
  if constexpr (DIM == -1 && RED != RED_NONE) finish_full<C, RED>(p, acc, smem);
}

// ---------------------------------------------------------------------------
// tilev: vectorised variant of tile for trees without a dim reduction.
//   Tile of TM = 32 V rows x 32 columns; thread (tx, ty) owns rows
//   32 V ti + V tx .. + V-1 of columns 32 tj + ty + 8 w (w < 4), so direct
//   reads and the output move V elements (16 bytes) per access.  A transposed
//   slot's 32 x TM source block is read with consecutive threads on
//   consecutive source rows into stage[q][column][row] (row stride TM + 4, a
//   multiple of 16 bytes) and read back as one 16-byte vector per thread.
// ---------------------------------------------------------------------------
// V values of the compute type from 16-byte aligned shared memory, one
// 16-byte access per 16 bytes
struct __align__(16) W4 {
  u32 w[4];
};
template <class C> struct FromWords;
template <> struct FromWords<float> {
  static constexpr int per = 4;
  __device__ static float get(const u32* w, int l) { return __uint_as_float(w[l]); }
};
template <> struct FromWords<int> {
  static constexpr int per = 4;
  __device__ static int get(const u32* w, int l) { return (int)w[l]; }
};
template <> struct FromWords<double> {
  static constexpr int per = 2;
  __device__ static double get(const u32* w, int l) { return __hiloint2double((int)w[2 * l + 1], (int)w[2 * l]); }
};
template <class C, int V> __device__ __forceinline__ void lds_vec(const C* p, C (&v)[V]) {
  constexpr int PER = FromWords<C>::per;
  static_assert(V % PER == 0, "whole 16-byte groups");
  const W4* q = reinterpret_cast<const W4*>(p);
#pragma unroll
  for (int n = 0; n < V / PER; ++n) {
    W4 t = q[n];
#pragma unroll
    for (int l = 0; l < PER; ++l) v[n * PER + l] = FromWords<C>::get(t.w, l);
  }
}

template <class T, class S, int NS, int NK, int RED, int TRMASK, bool OUT, int V>
__device__ __forceinline__ void tilev_kernel(const Params& p) {
  typedef typename ctype<S>::type C;
  typedef typename AccSel<C, RED>::type A;
  constexpr int NTR = popc<TRMASK>::value;
  constexpr int TM = TILE * V;
  constexpr int SP = TM + 16 / (int)sizeof(C);
  __shared__ __align__(16) C stage[NTR > 0 ? NTR : 1][TILE][SP];
  __shared__ A smem[32];
  Scal<C, NK> k;
#pragma unroll
  for (int q = 0; q < NK; ++q) k.k[q] = scalar_from_bits<C>(p.k[q]);
  typename CsqOf<C>::type csq;
  if constexpr (RED == RED_CSQ) csq.set_mean(*p.mu);
  u32 err = 0;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const long long nr = p.n_rows, nc = p.n_cols;
  const long long ntr = (nr + TM - 1) / TM, ntc = (nc + TILE - 1) / TILE;
  const long long tiles = ntr * ntc;
  A accs[V];
#pragma unroll
  for (int l = 0; l < V; ++l) accs[l].init();
  for (long long t = blockIdx.x; t < tiles; t += gridDim.x) {
    const long long ti = t % ntr, tj = t / ntr;
    const long long i0 = ti * TM + (long long)tx * V;
    const bool fullr = (i0 + V <= nr);
    Vals<C, NS, V> x[TILE_Q];
    // direct reads first: in flight while transposed blocks are staged
#pragma unroll
    for (int w = 0; w < TILE_Q; ++w) {
      const long long j = tj * TILE + ty + TILE_PH * w;
#pragma unroll
      for (int s = 0; s < NS; ++s) {
        if ((TRMASK >> s) & 1) continue;
        if (j < nc && fullr) {
          IO<S>::template load<V>(at<S>(p.src[s], i0, j, p.ld[s]), x[w].v[s]);
        } else {
#pragma unroll
          for (int l = 0; l < V; ++l)
            x[w].v[s][l] = (j < nc && i0 + l < nr) ? IO<S>::load1(at<S>(p.src[s], i0 + l, j, p.ld[s])) : C(0);
        }
      }
    }
    if constexpr (NTR > 0) {
      __syncthreads();  // the previous tile's shared reads are done
      int q = 0;
#pragma unroll
      for (int s = 0; s < NS; ++s)
        if ((TRMASK >> s) & 1) {
          const long long vr = tj * TILE + tx;  // view row = output column
          C v[TM / TILE_PH];  // all of this thread's staging loads in flight at once
#pragma unroll
          for (int u = 0; u < TM / TILE_PH; ++u) {
            const long long vc = ti * TM + ty + TILE_PH * u;  // view column = output row
            v[u] = (vr < nc && vc < nr) ? IO<S>::load1(at<S>(p.src[s], vr, vc, p.ld[s])) : C(0);
          }
#pragma unroll
          for (int u = 0; u < TM / TILE_PH; ++u) stage[q][tx][ty + TILE_PH * u] = v[u];
          ++q;
        }
      __syncthreads();
      q = 0;
#pragma unroll
      for (int s = 0; s < NS; ++s)
        if ((TRMASK >> s) & 1) {
#pragma unroll
          for (int w = 0; w < TILE_Q; ++w) lds_vec<C, V>(&stage[q][ty + TILE_PH * w][tx * V], x[w].v[s]);
          ++q;
        }
    }
#pragma unroll
    for (int w = 0; w < TILE_Q; ++w) {
      const long long j = tj * TILE + ty + TILE_PH * w;
      if (j >= nc) continue;
      if (fullr) {
        C y[V];
#pragma unroll
        for (int l = 0; l < V; ++l) y[l] = eval_elem<T, RED>(x[w], k, err, l, accs[l], csq, i0 + l + j * nr);
        if constexpr (OUT) IO<S>::template store<V>(at_out<S>(p.out, i0, j, p.out_ld), y);
      } else {
#pragma unroll
        for (int l = 0; l < V; ++l)
          if (i0 + l < nr) {
            C y = eval_elem<T, RED>(x[w], k, err, l, accs[l], csq, i0 + l + j * nr);
            if constexpr (OUT) IO<S>::store1(at_out<S>(p.out, i0 + l, j, p.out_ld), y);
          }
      }
    }
  }
  if (err) atomicOr(p.err_flag, err);
  if constexpr (RED != RED_NONE) {
#pragma unroll
    for (int l = 1; l < V; ++l) accs[0].merge(accs[l]);
    finish_full<C, RED>(p, accs[0], smem);
  }
}

// ---------------------------------------------------------------------------
// adj: gradient of L = mult * sum(tree) with respect to every slot
// ---------------------------------------------------------------------------
template <class T, class S, int NS, int NK, int V, int U>
__device__ __forceinline__ void adj_kernel(const Params& p) {
  typedef typename ctype<S>::type C;
  Scal<C, NK> k;
#pragma unroll
  for (int q = 0; q < NK; ++q) k.k[q] = scalar_from_bits<C>(p.k[q]);
  u32 err = 0;
  const C g0 = (C)((double)(*(const C*)p.upstream) * p.grad_mult);
  const long long nr = p.n_rows, nc = p.n_cols, cpc = p.units_per_col;
  const long long units = cpc * nc;
  const long long step = (long long)blockDim.x * V;
  const long long CH = step * U;
  for (long long u = blockIdx.x; u < units; u += gridDim.x) {
    const long long j = (nc == 1) ? 0 : u / cpc;
    const long long i0 = (u - j * cpc) * CH + (long long)threadIdx.x * V;
    Vals<C, NS, V> x[U];
    bool full[U];
#pragma unroll
    for (int g = 0; g < U; ++g) {
      const long long i = i0 + g * step;
      full[g] = (i + V <= nr);
      if (full[g]) {
#pragma unroll
        for (int s = 0; s < NS; ++s) IO<S>::template load<V>(at<S>(p.src[s], i, j, p.ld[s]), x[g].v[s]);
      } else {
#pragma unroll
        for (int s = 0; s < NS; ++s)
#pragma unroll
          for (int l = 0; l < V; ++l) x[g].v[s][l] = (i + l < nr) ? IO<S>::load1(at<S>(p.src[s], i + l, j, p.ld[s])) : C(0);
      }
    }
#pragma unroll
    for (int g = 0; g < U; ++g) {
      const long long i = i0 + g * step;
      C gs[NS][V];
#pragma unroll
      for (int l = 0; l < V; ++l) {
        C gl[NS];
#pragma unroll
        for (int s = 0; s < NS; ++s) gl[s] = C(0);
        if (full[g] || i + l < nr) T::bw(x[g], k, err, l, g0, gl);
#pragma unroll
        for (int s = 0; s < NS; ++s) gs[s][l] = gl[s];
      }
#pragma unroll
      for (int s = 0; s < NS; ++s) {
        if (p.grad[s] == nullptr) continue;
        if (full[g]) {
          IO<S>::template store<V>(at_out<S>(p.grad[s], i, j, p.grad_ld[s]), gs[s]);
        } else {
#pragma unroll
          for (int l = 0; l < V; ++l)
            if (i + l < nr) IO<S>::store1(at_out<S>(p.grad[s], i + l, j, p.grad_ld[s]), gs[s][l]);
        }
      }
    }
  }
  if (err) atomicOr(p.err_flag, err);
}

// ---------------------------------------------------------------------------
// batch: persistent kernel over the 32x32 tiles of many problems, one warp
// per tile.  Every warp takes `chunk` consecutive tiles at a time from an
// atomic queue (the next pop is issued before the current chunk is worked
// on, so its latency is hidden) and synchronises only with itself: a
// transposed read goes through the warp's own padded shared-memory tile.
// A problem's tiles inside one chunk are accumulated in registers and
// flushed once -- a problem whose tiles all lie in one chunk writes its
// result directly; otherwise each flush leaves one partial per tile range and
// the flush that completes the problem combines its partials in tile order.
// Chunks start at multiples of `chunk`, so the grouping -- and the result --
// does not depend on which warp took which chunk.
// ---------------------------------------------------------------------------
constexpr int BATCH_WARPS = 8;  // warps per block when shared memory allows
constexpr int BATCH_COLS = 16;  // tile columns loaded per step

// warps per block: each warp owns NTR padded tiles of the compute type, and
// the block's static shared memory stays within 48 KiB (the host launches
// blockDim.x = 32 * batch_warps)
template <int NTR, int CSIZE> struct BatchWarps {
  static constexpr int per = TILE * (TILE + 1) * CSIZE * (NTR > 0 ? NTR : 1);
  static constexpr int fit = 49152 / per;
  static constexpr int value = NTR == 0 ? BATCH_WARPS : (fit < 1 ? 1 : (fit > BATCH_WARPS ? BATCH_WARPS : fit));
};

template <class C, class A>
__device__ __forceinline__ void batch_write(const BatchParams& bp, long long p, const A& a, long long count) {
  typedef typename rtype<C>::type R;
  if constexpr (is_int_c<C>::value) {
    ((long long*)bp.red_out)[p] = a.ivalue();
  } else {
    double v = a.value();
    if (bp.mean) v /= (double)count;
    ((R*)bp.red_out)[p] = (R)v;
  }
}

template <class C, class A>
__device__ __forceinline__ void batch_flush(const BatchParams& bp, long long p, long long ta, long long tb, A acc) {
  const int lane = threadIdx.x & 31;
  acc = warp_reduce(acc);  // every lane holds the sum
  const BatchProblem& pr = bp.probs[p];
  const long long ntile = bp.tile_begin[p + 1] - pr.tile_begin;
  const long long count = pr.n_rows * pr.n_cols;
  if (tb - ta == ntile) {  // the whole problem is in this group
    if (lane == 0) batch_write<C>(bp, p, acc, count);
    return;
  }
  A zero;
  zero.init();
  for (long long t = ta + 1 + lane; t < tb; t += 32) ((A*)bp.partials)[t] = zero;
  if (lane == 0) ((A*)bp.partials)[ta] = acc;
  __threadfence();
  __syncwarp();
  unsigned int d = 0;
  if (lane == 0) d = atomicAdd(&bp.done[p], (unsigned int)(tb - ta));
  d = __shfl_sync(0xffffffffu, d, 0);
  if ((long long)d + (tb - ta) == ntile) {
    __threadfence();
    A a;
    a.init();
    for (long long s = lane; s < ntile; s += 32) a.merge(load_cg(&((const A*)bp.partials)[pr.tile_begin + s]));
    a = warp_reduce(a);
    if (lane == 0) {
      batch_write<C>(bp, p, a, count);
      bp.done[p] = 0u;
    }
  }
}

template <class T, class S, int NS, int NK, int TRMASK, bool RED>
__device__ __forceinline__ void batch_kernel(const BatchParams bp) {
  typedef typename ctype<S>::type C;
  typedef typename AccOf<C>::type A;
  constexpr int NTR = popc<TRMASK>::value;
  constexpr int BW = BatchWarps<NTR, (int)sizeof(C)>::value;
  __shared__ C stage_all[BW][NTR > 0 ? NTR : 1][TILE][TILE + 1];
  Scal<C, NK> k;
#pragma unroll
  for (int q = 0; q < NK; ++q) k.k[q] = scalar_from_bits<C>(bp.k[q]);
  typename CsqOf<C>::type csq;
  u32 err = 0;
  const int tx = threadIdx.x & 31, wid = threadIdx.x >> 5;
  C (*stage)[TILE][TILE + 1] = stage_all[wid];
  unsigned int pop = 0;
  if (tx == 0) pop = atomicAdd(&bp.queue[0], (unsigned int)bp.chunk);
  long long t0 = (long long)__shfl_sync(0xffffffffu, pop, 0);
  while (t0 < bp.n_tiles) {
    unsigned int nxt = 0;
    if (tx == 0) nxt = atomicAdd(&bp.queue[0], (unsigned int)bp.chunk);  // used after the chunk
    const long long t1 = (t0 + bp.chunk < bp.n_tiles) ? t0 + bp.chunk : bp.n_tiles;
    // the chunk's owning problems, one lane per tile (chunk <= 32)
    const int myp = (t0 + tx < t1) ? bp.tile_prob[t0 + tx] : 0;
    A acc;
    acc.init();
    long long cur = -1, gfirst = t0;
    for (long long t = t0; t < t1; ++t) {
      const long long p = __shfl_sync(0xffffffffu, myp, (int)(t - t0));
      if constexpr (RED) {
        if (p != cur && cur >= 0) {
          batch_flush<C>(bp, cur, gfirst, t, acc);
          acc.init();
          gfirst = t;
        }
      }
      cur = p;
      // the problem record in registers: the tile's stores to Y could alias
      // it as far as the compiler knows, which would reload every field
      const BatchProblem pr = bp.probs[p];
      const long long nr = pr.n_rows, nc = pr.n_cols;
      const long long lt = t - pr.tile_begin;
      const long long ti = lt % pr.n_tile_rows, tj = lt / pr.n_tile_rows;
      const long long r0 = ti * TILE, c0 = tj * TILE;
      const int nrows = (int)((nr - r0 < TILE) ? nr - r0 : TILE);  // warp-uniform extents
      const int ncols = (int)((nc - c0 < TILE) ? nc - c0 : TILE);
      if constexpr (NTR > 0) {
        // stage the transposed blocks: view(c0 + tx, r0 + m) -> stage[q][m][tx]
        int q = 0;
#pragma unroll
        for (int s = 0; s < NS; ++s)
          if ((TRMASK >> s) & 1) {
            // 32 loads in flight per lane, then 32 shared stores
            for (int m0 = 0; m0 < nrows; m0 += 32) {
              C v[32];
#pragma unroll
              for (int u = 0; u < 32; ++u)
                v[u] = (tx < ncols && m0 + u < nrows) ? IO<S>::load1(at<S>(pr.src[s], c0 + tx, r0 + m0 + u, pr.ld[s]))
                                                      : C(0);
#pragma unroll
              for (int u = 0; u < 32; ++u)
                if (m0 + u < nrows) stage[q][m0 + u][tx] = v[u];
            }
            ++q;
          }
        __syncwarp();
      }
      const bool row_ok = tx < nrows;
      for (int jb = 0; jb < ncols; jb += BATCH_COLS) {
        Vals<C, NS, BATCH_COLS> x;
#pragma unroll
        for (int jj = 0; jj < BATCH_COLS; ++jj) {
          const bool ok = row_ok && (jb + jj < ncols);
          int q = 0;
#pragma unroll
          for (int s = 0; s < NS; ++s) {
            if ((TRMASK >> s) & 1) {
              x.v[s][jj] = ok ? stage[q][tx][jb + jj] : C(0);
              ++q;
            } else {
              x.v[s][jj] = ok ? IO<S>::load1(at<S>(pr.src[s], r0 + tx, c0 + jb + jj, pr.ld[s])) : C(0);
            }
          }
        }
#pragma unroll
        for (int jj = 0; jj < BATCH_COLS; ++jj) {
          if (row_ok && jb + jj < ncols) {
            C y = eval_elem<T, RED ? RED_SUM : RED_NONE>(x, k, err, jj, acc, csq, 0);
            if (bp.has_out) IO<S>::store1(at_out<S>(pr.out, r0 + tx, c0 + jb + jj, pr.out_ld), y);
          }
        }
      }
      if constexpr (NTR > 0) __syncwarp();  // stage reads done before the next tile
    }
    if constexpr (RED) {
      if (cur >= 0) batch_flush<C>(bp, cur, gfirst, t1, acc);
    }
    t0 = (long long)__shfl_sync(0xffffffffu, nxt, 0);
  }
  if (err) atomicOr(bp.err_flag, err);
  // the last warp out resets the queue for the next launch
  if (tx == 0) {
    unsigned int e = atomicAdd(&bp.queue[1], 1u);
    if (e == gridDim.x * (blockDim.x >> 5) - 1) {
      bp.queue[0] = 0u;
      bp.queue[1] = 0u;
    }
  }
}

}  // namespace coot
