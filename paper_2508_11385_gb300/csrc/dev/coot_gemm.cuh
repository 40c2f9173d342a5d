// coot_gemm.cuh -- op(A) * op(B) on the tensor cores with the tree fused
// onto the product (Sec. 3: trans(X)*Y maps onto one GEMM call with a
// transposed operand; the element-wise part of the expression is evaluated
// on the product before it is stored).  Two kernels: gemm_tc_kernel
// (tcgen05, further below) for every operand layout TMA can address, and
// gemm_kernel (mma.sync) for the rest.
//
// gemm_kernel: BF16 / FP16 operands, FP32 accumulation, mma.sync m16n8k16.  CTA tile
// 128 x 128 x 32, 8 warps as 2 (M) x 4 (N), warp tile 64 x 32.  Operand
// tiles go global -> shared with 16-byte cp.async (zero-filled past the
// edges), two stages, and shared -> registers with ldmatrix; a K-contiguous
// operand is stored [row][k] and loaded as is, an M- or N-contiguous one is
// stored [k][row] and loaded with ldmatrix.trans.  16-byte chunks are
// XOR-swizzled per row so that the eight row addresses of an ldmatrix fall
// on different bank groups.  The epilogue evaluates the tree on each product
// element in registers (the product is slot PS of the tree; the other slots
// are read at the same (i, j)) and writes Y.
#pragma once
#include "coot_kernels.cuh"

namespace coot {

constexpr int GEMM_BM = GEMM_TILE, GEMM_BN = GEMM_TILE, GEMM_BK = 32, GEMM_THREADS = 256;

template <class S> struct Mma;
template <> struct Mma<bf16> {
  __device__ static void run(float (&d)[4], const u32 (&a)[4], u32 b0, u32 b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
  }
};
template <> struct Mma<f16> {
  __device__ static void run(float (&d)[4], const u32 (&a)[4], u32 b0, u32 b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
  }
};

__device__ __forceinline__ u32 smem_u32(const void* p) { return (u32)__cvta_generic_to_shared(p); }

template <bool TRANS> __device__ __forceinline__ void ldsm_x4(u32 (&r)[4], u32 addr) {
  if constexpr (TRANS)
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(addr));
  else
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(addr));
}

// 16 bytes global -> shared, zero-filled when !ok (src is then not read)
__device__ __forceinline__ void cp_async16(u32 dst, const void* src, bool ok) {
  const int n = ok ? 16 : 0;
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(n));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;"); }
template <int N> __device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N)); }

// One operand tile in shared memory: ROWS x 32 (K-contiguous: rows are M or
// N, 4 chunks of 8 along K) or 32 x COLS (not K-contiguous: rows are K, the
// chunks run along M or N).  Chunk (r, c) lives at r * CPR + (c ^ swz(r)).
template <bool KCONT> struct TileLayout {
  static constexpr int CPR = KCONT ? GEMM_BK / 8 : GEMM_BM / 8;  // 16-byte chunks per row
  static constexpr int ROWS = KCONT ? GEMM_BM : GEMM_BK;
  __device__ static int swz(int r) { return KCONT ? ((r >> 1) & 3) : (r & 7); }
  __device__ static int chunk(int r, int c) { return r * CPR + (c ^ swz(r)); }
};

// global -> shared for one operand tile.  KCONT: element (row, k) of op(X) at
// X[k + row * ld]; else at X[row + k * ld].  row0/k0: tile origin; nrow/nk:
// extents of op(X).  16-byte cp.async when the whole chunk is inside and
// aligned, else element by element (zeros outside).
template <class S, bool KCONT>
__device__ __forceinline__ void load_tile(u32 sbase, const S* X, long long ld, long long row0, long long k0,
                                          long long nrow, long long nk, bool vec) {
  typedef TileLayout<KCONT> Lt;
  constexpr int NCH = Lt::ROWS * Lt::CPR;  // 512
#pragma unroll
  for (int q = 0; q < NCH / GEMM_THREADS; ++q) {
    const int ch = threadIdx.x + q * GEMM_THREADS;
    const int r = ch / Lt::CPR, c = ch % Lt::CPR;
    // the chunk's first element and the stride of its 8 elements
    long long orow, ok0;
    if constexpr (KCONT) {
      orow = row0 + r;
      ok0 = k0 + 8 * c;
    } else {
      orow = row0 + 8 * c;
      ok0 = k0 + r;
    }
    const u32 dst = sbase + 16u * (u32)Lt::chunk(r, c);
    const S* src = KCONT ? X + (ok0 + orow * ld) : X + (orow + ok0 * ld);
    const bool inside = KCONT ? (orow < nrow && ok0 + 8 <= nk) : (ok0 < nk && orow + 8 <= nrow);
    if (vec && inside) {
      cp_async16(dst, src, true);
    } else {
      // ragged edge or unaligned operand: element by element
      u16 e[8];
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        const bool ok = KCONT ? (orow < nrow && ok0 + t < nk) : (ok0 < nk && orow + t < nrow);
        e[t] = ok ? ldg_u16(src + t) : (u16)0;  // the 8 elements are adjacent in memory either way
      }
      const u32 w0 = (u32)e[0] | ((u32)e[1] << 16), w1 = (u32)e[2] | ((u32)e[3] << 16);
      const u32 w2 = (u32)e[4] | ((u32)e[5] << 16), w3 = (u32)e[6] | ((u32)e[7] << 16);
      asm volatile("st.shared.v4.u32 [%0], {%1,%2,%3,%4};" ::"r"(dst), "r"(w0), "r"(w1), "r"(w2), "r"(w3));
    }
  }
}

template <class T, class S, int NS, int NK, int PS, bool KA, bool KB>
__device__ __forceinline__ void gemm_kernel(const GemmParams& gp) {
  typedef float C;
  typedef TileLayout<KA> LA;
  typedef TileLayout<KB> LB;
  constexpr int A_BYTES = LA::ROWS * LA::CPR * 16, B_BYTES = LB::ROWS * LB::CPR * 16;
  __shared__ __align__(128) unsigned char smem[2][A_BYTES + B_BYTES];
  const Params& p = gp.p;
  const S* A = (const S*)gp.a;
  const S* B = (const S*)gp.b;
  const long long M = gp.m, N = gp.n, K = gp.k;
  const long long m0 = (long long)blockIdx.x * GEMM_BM, n0 = (long long)blockIdx.y * GEMM_BN;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int wm = warp & 1, wn = warp >> 1;  // warp tile: rows 64 wm.., cols 32 wn..
  const bool vec = gp.vec != 0;
  float acc[4][4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[a][b][c] = 0.f;

  const long long nkt = (K + GEMM_BK - 1) / GEMM_BK;
  auto stage_a = [&](int st) { return smem_u32(&smem[st][0]); };
  auto stage_b = [&](int st) { return smem_u32(&smem[st][A_BYTES]); };
  if (nkt > 0) {
    load_tile<S, KA>(stage_a(0), A, gp.lda, m0, 0, M, K, vec);
    load_tile<S, KB>(stage_b(0), B, gp.ldb, n0, 0, N, K, vec);
  }
  cp_async_commit();
  for (long long kt = 0; kt < nkt; ++kt) {
    const int st = (int)(kt & 1);
    if (kt + 1 < nkt) {
      load_tile<S, KA>(stage_a(st ^ 1), A, gp.lda, m0, (kt + 1) * GEMM_BK, M, K, vec);
      load_tile<S, KB>(stage_b(st ^ 1), B, gp.ldb, n0, (kt + 1) * GEMM_BK, N, K, vec);
    }
    cp_async_commit();
    cp_async_wait<1>();  // this stage's group has landed
    __syncthreads();
    const u32 sa = stage_a(st), sb = stage_b(st);
#pragma unroll
    for (int kk = 0; kk < GEMM_BK; kk += 16) {
      // A fragments: four 16 x 16 tiles of the warp's 64 rows
      u32 af[4][4];
      const int mat = lane >> 3, r8 = lane & 7;
#pragma unroll
      for (int mt = 0; mt < 4; ++mt) {
        const int mrow = wm * 64 + mt * 16;
        int rr, cc;
        if constexpr (KA) {  // [m][k]: rows m, chunks along k
          rr = mrow + r8 + (mat & 1) * 8;
          cc = kk / 8 + (mat >> 1);
        } else {  // [k][m]: rows k, chunks along m
          rr = kk + r8 + (mat >> 1) * 8;
          cc = (mrow + (mat & 1) * 8) / 8;
        }
        ldsm_x4<!KA>(af[mt], sa + 16u * (u32)LA::chunk(rr, cc));
      }
      // B fragments: four 16 x 8 tiles of the warp's 32 columns, two per ldmatrix
      u32 bf[4][2];
#pragma unroll
      for (int np = 0; np < 2; ++np) {
        const int ncol = wn * 32 + np * 16;
        int rr, cc;
        u32 t[4];
        if constexpr (KB) {  // [n][k]
          rr = ncol + r8 + (mat >> 1) * 8;
          cc = kk / 8 + (mat & 1);
        } else {  // [k][n]
          rr = kk + r8 + (mat & 1) * 8;
          cc = (ncol + (mat >> 1) * 8) / 8;
        }
        ldsm_x4<!KB>(t, sb + 16u * (u32)LB::chunk(rr, cc));
        bf[2 * np][0] = t[0];
        bf[2 * np][1] = t[1];
        bf[2 * np + 1][0] = t[2];
        bf[2 * np + 1][1] = t[3];
      }
#pragma unroll
      for (int mt = 0; mt < 4; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) Mma<S>::run(acc[mt][nt], af[mt], bf[nt][0], bf[nt][1]);
    }
    __syncthreads();  // the stage is free for the load two steps ahead
  }
  cp_async_wait<0>();

  // epilogue: the tree on every product element of the warp tile
  Scal<C, NK> k;
#pragma unroll
  for (int q = 0; q < NK; ++q) k.k[q] = scalar_from_bits<C>(p.k[q]);
  u32 err = 0;
  const int g = lane >> 2, tq = lane & 3;
#pragma unroll
  for (int mt = 0; mt < 4; ++mt)
#pragma unroll
    for (int nt = 0; nt < 4; ++nt)
#pragma unroll
      for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const long long i = m0 + wm * 64 + mt * 16 + g + 8 * h;
          const long long j = n0 + wn * 32 + nt * 8 + 2 * tq + e;
          if (i < M && j < N) {
            Vals<C, NS, 1> x;
#pragma unroll
            for (int s = 0; s < NS; ++s)
              x.v[s][0] = (s == PS) ? acc[mt][nt][2 * h + e] : IO<S>::load1(at_slot<S>(p, s, i, j));
            const C y = T::ev(x, k, err, 0);
            IO<S>::store1(at_out_g<S>(p, i, j), y);
          }
        }
  if (err) atomicOr(p.err_flag, err);
}

// ---------------------------------------------------------------------------
// The same GEMM on the 5th-generation tensor cores (tcgen05), for every
// operand layout: an operand with K adjacent (op(A) of trans(X), op(B) of
// Y) is "K-major", one with M or N adjacent "MN-major".
//   Persistent: one CTA per SM (192 KiB of operand stages) walks output
//   tiles of 256 x 256, 320 threads in three roles:
//   * warp 0, one thread: TMA loads of the operand tiles (64 K values x 256
//     rows each, 128-byte swizzle) into a 3-stage ring; it waits for a
//     stage's "empty" barrier and announces the stage's bytes on its "full"
//     barrier.  K-major: one box per operand, each tile row 64 K values =
//     128 bytes, 8-row groups forming 1 KiB swizzle atoms -- the K-major
//     SWIZZLE_128B layout of the MMA (1 KiB between 8-row groups; a K = 16
//     step moves the start address 32 bytes).  MN-major: boxes of 64 rows
//     (128 bytes, the adjacent dimension) x 64 K values, one per 64 rows of
//     the tile, 8 KiB apart -- the MN-major SWIZZLE_128B layout (8 KiB
//     between 64-row blocks, 1 KiB between groups of 8 K values; a K = 16
//     step moves the start address 2 KiB).  Either way the tile's rows
//     128-255 start 16 KiB after its rows 0-127.  TMA fills rows and K
//     values past the matrix with zeros, so ragged m, n and k need no
//     special case.
//   * warp 1, one thread: waits for "full" and issues, per K = 16 step, two
//     M = 128, N = 256 MMAs sharing the B tile: rows 0-127 into accumulator
//     columns 0-255 and rows 128-255 into columns 256-511 (FP32 in tensor
//     memory, lane = row within the half); it commits each stage to its
//     "empty" barrier and the tile's last step to "acc full".  A 256 x 256
//     tile does 128 FLOP per operand byte staged (a 128 x 256 tile 85), so
//     the three stages hold 1.5x the MMA work of four 128 x 256 stages in
//     the same shared memory -- the ring's depth against the TMA round trip
//     is what bounded the smaller tile.  The accumulator fills tensor
//     memory, so a tile's MMAs start once the epilogue has drained the
//     previous tile ("acc empty"); the producer keeps loading meanwhile.
//   * warps 2-9, the epilogue: warp w reads lanes 32 (w % 4).. (rows) of
//     each half of the accumulator -- columns 0-127 for warps 2-5, 128-255
//     for warps 6-9 -- 32 or 16 columns at a time, loads the
//     tree's other leaves at the same (i, j) ahead of the tensor-memory read,
//     applies the tree and stores Y (consecutive lanes: consecutive rows of
//     the column-major result); it then releases the accumulator.
//   Tiles are numbered in groups of 16 tile rows (M), N-major inside a
//   group, and CTA b takes tiles b, b + grid, ...: the tiles in flight share
//   their A and B tiles in L2.
//   Every wait is bounded by the global timer (2 s): past it the thread
//   raises device flag COOT_FLAG_WAIT_TIMEOUT (results are then undefined)
//   and its remaining waits give up at once; tensor memory is always
//   released.  A launch whose barriers never complete therefore ends after
//   one 2 s wait per thread.
// ---------------------------------------------------------------------------
constexpr int TC_BM = GEMM_TC_BM, TC_BN = GEMM_TC_BN, TC_BK = GEMM_TC_BK, TC_ST = GEMM_TC_STAGES;
constexpr int TC_A_BYTES = TC_BM * TC_BK * 2, TC_B_BYTES = TC_BN * TC_BK * 2;
constexpr int TC_BAR_OFF = TC_ST * (TC_A_BYTES + TC_B_BYTES);
constexpr int TC_GROUP_M = 16;
constexpr unsigned long long TC_WAIT_NS = 2000000000ull;  // 2 s

template <class S> struct TcFmt;
template <> struct TcFmt<bf16> { static constexpr u32 v = 1; };
template <> struct TcFmt<f16> { static constexpr u32 v = 0; };

// shared-memory matrix descriptor, 128-byte swizzle.  K-major: 1 KiB
// between 8-row groups (the leading byte offset is not used).  MN-major:
// leading byte offset 8 KiB between 64-row blocks, stride byte offset 1 KiB
// between groups of 8 K values.
template <bool KMAJ> __device__ __forceinline__ unsigned long long tc_desc(u32 saddr) {
  const unsigned long long start = (saddr >> 4) & 0x3FFFull;
  const unsigned long long lbo = KMAJ ? 1 : (8192u >> 4), sbo = 1024u >> 4;
  return start | (lbo << 16) | (sbo << 32) | (1ull << 46) | (2ull << 61);  // version 1; SWIZZLE_128B
}
// start-address step of one K = 16 MMA, in the descriptor's 16-byte units
template <bool KMAJ> __device__ constexpr unsigned long long tc_kstep() { return KMAJ ? 32u >> 4 : 2048u >> 4; }
// instruction descriptor of kind::f16: FP32 accumulator, A and B of the
// storage type, M = 128, N = 256; bits 15 / 16 mark an MN-major A / B
template <class S, bool KA, bool KB> __device__ __forceinline__ u32 tc_idesc() {
  return (1u << 4) | (TcFmt<S>::v << 7) | (TcFmt<S>::v << 10) | ((KA ? 0u : 1u) << 15) | ((KB ? 0u : 1u) << 16) |
         ((u32)(TC_BN >> 3) << 17) | ((u32)(GEMM_TC_MMA_M >> 4) << 24);
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// a thread's bounded waits: wait until the barrier's phase of the given
// parity has completed, at most TC_WAIT_NS; once one wait has failed
// (`dead`), later ones only probe
struct TcWait {
  bool dead;
  u32 err;
  __device__ void operator()(u32 mbar, u32 parity) {
    const unsigned long long t0 = global_ns();
    for (unsigned it = 0;; ++it) {
      u32 done;
      asm volatile(
          "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
          : "=r"(done)
          : "r"(mbar), "r"(parity)
          : "memory");
      if (done) return;
      if ((it & 63) == 63 && (dead || global_ns() - t0 > TC_WAIT_NS)) {
        dead = true;
        err |= 2u;
        return;
      }
    }
  }
};

// TMA: box (k0.., row0..) of a K x rows tensor into shared memory, completing
// its bytes on mbar
__device__ __forceinline__ void tma_load_2d(u32 dst, const void* map, int k0, int row0, u32 mbar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          dst),
      "l"(map), "r"(k0), "r"(row0), "r"(mbar)
      : "memory");
}

__device__ __forceinline__ void tc_tile_origin(const GemmParams& gp, long long tile, long long& m0, long long& n0) {
  const long long per_group = (long long)TC_GROUP_M * gp.tiles_n;
  const long long first_m = (tile / per_group) * TC_GROUP_M;
  const long long gm = (gp.tiles_m - first_m) < TC_GROUP_M ? (gp.tiles_m - first_m) : TC_GROUP_M;
  m0 = (first_m + (tile % per_group) % gm) * TC_BM;
  n0 = ((tile % per_group) / gm) * TC_BN;
}

template <int W> __device__ __forceinline__ void tmem_ld(u32 taddr, u32 (&v)[W]);
template <> __device__ __forceinline__ void tmem_ld<16>(u32 taddr, u32 (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
        "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(taddr));
}
template <> __device__ __forceinline__ void tmem_ld<32>(u32 taddr, u32 (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,"
      "%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
        "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]),
        "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
        "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr));
}

// one operand tile of a stage: ROWS rows from row0, K values from k0
template <bool KMAJ, int ROWS>
__device__ __forceinline__ void tc_load_operand(u32 dst, const void* map, int k0, int row0, u32 mbar) {
  if constexpr (KMAJ) {
    tma_load_2d(dst, map, k0, row0, mbar);
  } else {
#pragma unroll
    for (int b = 0; b < ROWS / 64; ++b) tma_load_2d(dst + 8192u * b, map, row0 + 64 * b, k0, mbar);
  }
}

template <class T, class S, int NS, int NK, int PS, bool KA, bool KB>
__device__ __forceinline__ void gemm_tc_kernel(const GemmParams& gp) {
  typedef float C;
  constexpr int W = NS <= 3 ? 32 : 16;  // accumulator columns per epilogue step
  extern __shared__ unsigned char tc_dyn[];
  const Params& p = gp.p;
  const long long M = gp.m, N = gp.n, K = gp.k;
  const long long n_tiles = gp.tiles_m * gp.tiles_n;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const u32 sbase = (smem_u32(tc_dyn) + 1023u) & ~1023u;
  const u32 full0 = sbase + TC_BAR_OFF, empty0 = full0 + 8 * TC_ST;
  const u32 afull0 = empty0 + 8 * TC_ST, aempty0 = afull0 + 16, tslot = aempty0 + 16;
  // the A tile's two halves of 128 rows: K-major, 128 rows of 128 bytes; MN-major,
  // two boxes of 64 rows (8 KiB each) -- 16 KiB apart either way
  constexpr u32 A_HALF = 16384;
  TcWait wait{false, 0};
  if (threadIdx.x == 0) {
    for (int st = 0; st < TC_ST; ++st) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(full0 + 8 * st));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(empty0 + 8 * st));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(afull0));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(aempty0), "n"(GEMM_TC_THREADS - 64));
    asm volatile("fence.mbarrier_init.release.cluster;");
    asm volatile("prefetch.tensormap [%0];" ::"l"(gp.tma_a) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(gp.tma_b) : "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tslot), "r"(2 * TC_BN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  u32 tmem;
  asm volatile("ld.shared.u32 %0, [%1];" : "=r"(tmem) : "r"(tslot) : "memory");

  const int nkt = (int)((K + TC_BK - 1) / TC_BK);
  if (warp == 0) {
    if (lane == 0) {
      // producer: one ring position per K step, across tiles
      unsigned it = 0;
      for (long long tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        long long m0, n0;
        tc_tile_origin(gp, tile, m0, n0);
        for (int kt = 0; kt < nkt; ++kt, ++it) {
          const int st = (int)(it % TC_ST);
          wait(empty0 + 8 * st, ((it / TC_ST) & 1u) ^ 1u);  // the first pass finds every stage empty
          const u32 fb = full0 + 8 * st;
          asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb),
                       "r"(TC_A_BYTES + TC_B_BYTES)
                       : "memory");
          tc_load_operand<KA, TC_BM>(sbase + (u32)(st * TC_A_BYTES), gp.tma_a, kt * TC_BK, (int)m0, fb);
          tc_load_operand<KB, TC_BN>(sbase + (u32)(TC_ST * TC_A_BYTES + st * TC_B_BYTES), gp.tma_b, kt * TC_BK,
                                     (int)n0, fb);
        }
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {
      // MMA issue: per K = 16 step, rows 0-127 of the tile into accumulator
      // columns 0-255 and rows 128-255 into columns 256-511, both with the
      // whole B tile
      const u32 idesc = tc_idesc<S, KA, KB>();
      unsigned it = 0, lt = 0;
      for (long long tile = blockIdx.x; tile < n_tiles; tile += gridDim.x, ++lt) {
        wait(aempty0, (lt & 1u) ^ 1u);  // the epilogue has drained the accumulator
        asm volatile("tcgen05.fence::after_thread_sync;");
        for (int kt = 0; kt < nkt; ++kt, ++it) {
          const int st = (int)(it % TC_ST);
          wait(full0 + 8 * st, (it / TC_ST) & 1u);
          asm volatile("tcgen05.fence::after_thread_sync;");
          const u32 abase = sbase + (u32)(st * TC_A_BYTES);
          const unsigned long long ad0 = tc_desc<KA>(abase);
          const unsigned long long ad1 = tc_desc<KA>(abase + A_HALF);
          const unsigned long long bd = tc_desc<KB>(sbase + (u32)(TC_ST * TC_A_BYTES + st * TC_B_BYTES));
#pragma unroll
          for (int kk = 0; kk < TC_BK / 16; ++kk) {
            const u32 accum = (kt > 0 || kk > 0) ? 1u : 0u;
            asm volatile(
                "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                "l"(ad0 + tc_kstep<KA>() * kk), "l"(bd + tc_kstep<KB>() * kk), "r"(idesc), "r"(accum));
            asm volatile(
                "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem + (u32)TC_BN),
                "l"(ad1 + tc_kstep<KA>() * kk), "l"(bd + tc_kstep<KB>() * kk), "r"(idesc), "r"(accum));
          }
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                           empty0 + 8 * st)
                       : "memory");
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(afull0)
                     : "memory");
      }
    }
    __syncwarp();
  } else {
    // epilogue: the tile's two halves of rows, each from its 256 accumulator
    // columns; warp w takes lane quarter w % 4 and columns 128 (w - 2) / 4 ..
    Scal<C, NK> k;
#pragma unroll
    for (int q = 0; q < NK; ++q) k.k[q] = scalar_from_bits<C>(p.k[q]);
    const int quarter = warp & 3;
    const int c0 = (TC_BN / 2) * ((warp - 2) >> 2);
    unsigned lt = 0;
    for (long long tile = blockIdx.x; tile < n_tiles; tile += gridDim.x, ++lt) {
      long long m0, n0;
      tc_tile_origin(gp, tile, m0, n0);
      wait(afull0, lt & 1u);
      __syncwarp();
      asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll 1
      for (int half = 0; half < 2; ++half) {
        const long long i = m0 + GEMM_TC_MMA_M * half + 32 * quarter + lane;
        if (m0 + GEMM_TC_MMA_M * half >= M) break;  // warp-uniform
#pragma unroll 1
        for (int cc = c0 / W; cc < (c0 + TC_BN / 2) / W; ++cc) {
          if (n0 + W * cc >= N) break;  // warp-uniform
          // the other leaves first, then the accumulator
          Vals<C, NS, 1> x[W];
#pragma unroll
          for (int t = 0; t < W; ++t) {
            const long long j = n0 + W * cc + t;
#pragma unroll
            for (int s2 = 0; s2 < NS; ++s2)
              if (s2 != PS) x[t].v[s2][0] = (i < M && j < N) ? IO<S>::load1(at_slot<S>(p, s2, i, j)) : C(0);
          }
          u32 v[W];
          tmem_ld<W>(tmem + (u32)(TC_BN * half) + ((u32)(32 * quarter) << 16) + (u32)(W * cc), v);
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
          for (int t = 0; t < W; ++t) {
            const long long j = n0 + W * cc + t;
            x[t].v[PS][0] = __uint_as_float(v[t]);
            const C y = T::ev(x[t], k, wait.err, 0);
            if (i < M && j < N) IO<S>::store1(at_out_g<S>(p, i, j), y);
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;");
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(aempty0) : "memory");
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * TC_BN));
  if (wait.err) atomicOr(p.err_flag, wait.err);
}

// ---------------------------------------------------------------------------
// The same GEMM for FP32 and FP64 operands on the CUDA cores (no tensor-core
// kind computes them exactly): accumulation in the storage type with fused
// multiply-adds, the same epilogue.
//   256 threads as 16 x 16, each owning TM x TN outputs (8 x 8 for FP32 in a
//   128 x 128 tile, 4 x 4 for FP64 in 64 x 64) as two halves of rows (and of
//   columns) half a tile apart, so that each fragment is read from shared
//   memory as 16-byte vectors with the 16 lanes of a half-warp on adjacent
//   chunks (no bank conflict).  Per K step of 16, the A and B
//   tiles are read from global memory into registers (threads walk the
//   operand's adjacent dimension, zeros past the edges), stored to shared
//   memory as [k][row] (rows padded by 4 so the stores of a K-adjacent
//   operand do not collide on a bank), and the next step's reads are issued
//   before this step's products, over two shared buffers.
// ---------------------------------------------------------------------------
template <class S> struct SimtCfg;
template <> struct SimtCfg<float> { static constexpr int BM = 128, BN = 128, TM = 8, TN = 8; };
template <> struct SimtCfg<double> { static constexpr int BM = 64, BN = 64, TM = 4, TN = 4; };
constexpr int SIMT_BK = 16, SIMT_THREADS = 256;

__device__ __forceinline__ float simt_fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double simt_fma(double a, double b, double c) { return __fma_rn(a, b, c); }

// element (row, k) of op(X): K adjacent -> X[k + row * ld], else X[row + k * ld]
template <class S, bool KMAJ, int ROWS>
__device__ __forceinline__ void simt_fetch(S (&r)[ROWS * SIMT_BK / SIMT_THREADS], const S* X, long long ld,
                                           long long row0, long long k0, long long nrow, long long nk) {
  constexpr int PER = ROWS * SIMT_BK / SIMT_THREADS;
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int idx = threadIdx.x + q * SIMT_THREADS;
    // walk the adjacent dimension with consecutive threads
    const int row = KMAJ ? idx / SIMT_BK : idx % ROWS;
    const int kk = KMAJ ? idx % SIMT_BK : idx / ROWS;
    const long long gr = row0 + row, gk = k0 + kk;
    r[q] = (gr < nrow && gk < nk) ? IO<S>::load1(KMAJ ? X + (gk + gr * ld) : X + (gr + gk * ld)) : S(0);
  }
}
template <class S, bool KMAJ, int ROWS>
__device__ __forceinline__ void simt_store(S (*sh)[ROWS + 4], const S (&r)[ROWS * SIMT_BK / SIMT_THREADS]) {
  constexpr int PER = ROWS * SIMT_BK / SIMT_THREADS;
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int idx = threadIdx.x + q * SIMT_THREADS;
    const int row = KMAJ ? idx / SIMT_BK : idx % ROWS;
    const int kk = KMAJ ? idx % SIMT_BK : idx / ROWS;
    sh[kk][row] = r[q];
  }
}

// position in the tile of a thread's i-th row (or column): halves of T/2
// at t * T/2 and TILE/2 + t * T/2
template <int T, int TILE_> __device__ __forceinline__ int simt_pos(int t, int i) {
  return (i < T / 2) ? t * (T / 2) + i : TILE_ / 2 + t * (T / 2) + (i - T / 2);
}
// a thread's T values of one shared row, as two 16-byte vectors
template <class S, int T, int TILE_> __device__ __forceinline__ void simt_frag(S (&v)[T], const S* row, int t);
template <> __device__ __forceinline__ void simt_frag<float, 8, 128>(float (&v)[8], const float* row, int t) {
  const float4 x = *(const float4*)(row + t * 4), y = *(const float4*)(row + 64 + t * 4);
  v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
  v[4] = y.x; v[5] = y.y; v[6] = y.z; v[7] = y.w;
}
template <> __device__ __forceinline__ void simt_frag<double, 4, 64>(double (&v)[4], const double* row, int t) {
  const double2 x = *(const double2*)(row + t * 2), y = *(const double2*)(row + 32 + t * 2);
  v[0] = x.x; v[1] = x.y; v[2] = y.x; v[3] = y.y;
}

template <class T, class S, int NS, int NK, int PS, bool KA, bool KB>
__device__ __forceinline__ void gemm_simt_kernel(const GemmParams& gp) {
  typedef SimtCfg<S> G;
  constexpr int BM = G::BM, BN = G::BN, TM = G::TM, TN = G::TN, BK = SIMT_BK;
  constexpr int PA = BM * BK / SIMT_THREADS, PB = BN * BK / SIMT_THREADS;
  __shared__ __align__(16) S As[2][BK][BM + 4];
  __shared__ __align__(16) S Bs[2][BK][BN + 4];
  const Params& p = gp.p;
  const S* A = (const S*)gp.a;
  const S* B = (const S*)gp.b;
  const long long M = gp.m, N = gp.n, K = gp.k;
  const long long m0 = (long long)blockIdx.x * BM, n0 = (long long)blockIdx.y * BN;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  S acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = S(0);
  const long long nkt = (K + BK - 1) / BK;
  S ra[PA], rb[PB];
  if (nkt > 0) {
    simt_fetch<S, KA, BM>(ra, A, gp.lda, m0, 0, M, K);
    simt_fetch<S, KB, BN>(rb, B, gp.ldb, n0, 0, N, K);
    simt_store<S, KA, BM>(As[0], ra);
    simt_store<S, KB, BN>(Bs[0], rb);
  }
  __syncthreads();
  for (long long kt = 0; kt < nkt; ++kt) {
    const int st = (int)(kt & 1);
    if (kt + 1 < nkt) {  // next step's reads in flight during this step's products
      simt_fetch<S, KA, BM>(ra, A, gp.lda, m0, (kt + 1) * BK, M, K);
      simt_fetch<S, KB, BN>(rb, B, gp.ldb, n0, (kt + 1) * BK, N, K);
    }
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      S a[TM], b[TN];
      simt_frag<S, TM, BM>(a, &As[st][kk][0], ty);
      simt_frag<S, TN, BN>(b, &Bs[st][kk][0], tx);
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = simt_fma(a[i], b[j], acc[i][j]);
    }
    if (kt + 1 < nkt) {
      simt_store<S, KA, BM>(As[st ^ 1], ra);
      simt_store<S, KB, BN>(Bs[st ^ 1], rb);
    }
    __syncthreads();
  }

  // epilogue: the tree on every product element of the thread's block
  typedef S C;
  Scal<C, NK> k;
#pragma unroll
  for (int q = 0; q < NK; ++q) k.k[q] = scalar_from_bits<C>(p.k[q]);
  u32 err = 0;
#pragma unroll
  for (int j = 0; j < TN; ++j)
#pragma unroll
    for (int i = 0; i < TM; ++i) {
      const long long gi = m0 + simt_pos<TM, BM>(ty, i), gj = n0 + simt_pos<TN, BN>(tx, j);
      if (gi < M && gj < N) {
        Vals<C, NS, 1> x;
#pragma unroll
        for (int s2 = 0; s2 < NS; ++s2)
          x.v[s2][0] = (s2 == PS) ? acc[i][j] : IO<S>::load1(at_slot<S>(p, s2, gi, gj));
        IO<S>::store1(at_out_g<S>(p, gi, gj), T::ev(x, k, err, 0));
      }
    }
  if (err) atomicOr(p.err_flag, err);
}

}  // namespace coot
