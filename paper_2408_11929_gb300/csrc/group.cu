// Grouped sweep steps (Section 2's block forward / backward substitution, reorganised).
//
// A grouped step writes several independent output lines at once ("tasks", see GTask in
// engine.h); each output line is a short sum of factor blocks times input lines,
//   out[out_line] = base + sum_q (+/-) F_{f_q} x_q,
// whose K ranges (node indices of the input lines) are concatenated.  The steps of the
// reorganised double sweep are of this form:
//   * the interface scans: a_s <- a_s + P a_{s -/+ 2^l} over all strips at once, P a power
//     of the strip transfer block (G for the forward pass, K for the backward pass);
//   * the corrections of the strips' interior lines: every line j of every strip in ONE step,
//     v_s[j] -= Y_j t_{s-1} (forward) and u_s[j] -= Z_j u_{s+1}[0] (backward), with stored
//     block columns Y_j = D^{-1}[j, 0] L and Z_j = D^{-1}[j, R-1] U of the strip inverse.
// Two kernels run them: complex64 with an even column count on the tensor cores
// (tc_group_kernel: TMA, tcgen05, tensor memory; K split summed in a thread-block cluster),
// otherwise on the CUDA cores (group_gemm_kernel, complex64 or complex128; K split summed by
// group_reduce_kernel).
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include <cudaTypedefs.h>

#include "common.cuh"
#include "engine.h"
#include "gemm.cuh"
#include "tc_gemm.cuh"

namespace hh {

// ------------------------------------------------------------------ CUDA-core form
// grid = (ceil(m / BM), total column tiles of the tasks, nsplit).  K split z covers stages
// [z kst, (z+1) kst) of the concatenated terms (each term ceil(m / BK) stages of BK nodes).
// With partial != nullptr the slices go to partial[(z m + row) totcols + coloff + col] for
// group_reduce_kernel, else the CTA applies the task's output rule itself.
template <typename R, int BM, int BN, int BK, int TM, int TN, int STAGES>
__global__ void __launch_bounds__(256) group_gemm_kernel(const typename Cx<R>::T* __restrict__ F, size_t blk, int lda,
                                                         int m, const GTask* __restrict__ tasks, int ntask, GArrays arrs,
                                                         int N, int C, int kst, typename Cx<R>::T* __restrict__ partial,
                                                         int totcols) {
  using T = typename Cx<R>::T;
  static_assert((BM / TM) * (BN / TN) == 256, "256 threads");
  constexpr int NTX = BN / TN;
  constexpr int ST_A = BM * BK, ST_B = BK * BN, ST = ST_A + ST_B;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* ring = reinterpret_cast<T*>(smem_raw);
  __shared__ GTask tk;
  __shared__ int s_tile, s_coloff;
  if (threadIdx.x == 0) {
    int by = blockIdx.y, ti = 0, coloff = 0;
    for (; ti < ntask - 1; ++ti) {
      const int cols = tasks[ti].ns * C, tiles = (cols + BN - 1) / BN;
      if (by < tiles) break;
      by -= tiles;
      coloff += cols;
    }
    tk = tasks[ti];
    s_tile = by;
    s_coloff = coloff;
  }
  __syncthreads();
  const int tid = threadIdx.x;
  const int tx = tid % NTX, ty = tid / NTX;
  const int row0 = blockIdx.x * BM;
  const int col0 = s_tile * BN;
  const int ncols = tk.ns * C;
  const int NC = N * C;
  const int spt = (m + BK - 1) / BK, nst = tk.nterm * spt;
  const int kb = blockIdx.z * kst, ke = min(nst, kb + kst);
  const int nk = ke > kb ? ke - kb : 0;

  auto issue = [&](int slot, int st) {
    T* As = ring + (size_t)slot * ST;
    T* Bs = As + ST_A;
    const int q = st / spt, k0 = (st % spt) * BK;
    const GTerm& g = tk.term[q];
    const T* A = F + (size_t)g.f * blk;
    for (int e = tid; e < BM * BK; e += 256) {
      const int r = e / BK, kk = e % BK;
      const int gr = row0 + r, gk = k0 + kk;
      const bool v = gr < m && gk < m;
      cp_async_elem(As + r * BK + kk, A + (size_t)(v ? gr : 0) * lda + (v ? gk : 0), v);
    }
    const T* X = reinterpret_cast<const T*>(arrs.p[g.arr]) + (size_t)g.line * m * NC;
    const int f0 = (tk.s0 + g.ds) * C + col0;  // flat (strip, column) index of the tile's first column
    for (int e = tid; e < BK * BN; e += 256) {
      const int kk = e / BN, cc = e % BN;
      const int gk = k0 + kk, fl = f0 + cc;
      const bool v = gk < m && col0 + cc < ncols && fl >= 0 && fl < NC;
      cp_async_elem(Bs + e, X + (v ? (size_t)gk * NC + fl : 0), v);
    }
  };

  R acc[TM][TN][2];
#pragma unroll
  for (int a = 0; a < TM; ++a)
#pragma unroll
    for (int b = 0; b < TN; ++b) acc[a][b][0] = acc[a][b][1] = 0;
#pragma unroll
  for (int s = 0; s < STAGES - 1; ++s) {
    if (s < nk) issue(s, kb + s);
    cp_async_commit();
  }
  for (int kt = 0; kt < nk; ++kt) {
    cp_async_wait<STAGES - 2>();
    __syncthreads();
    {
      const int nt = kt + STAGES - 1;
      if (nt < nk) issue(nt % STAGES, kb + nt);
      cp_async_commit();
    }
    const T* As = ring + (size_t)(kt % STAGES) * ST;
    const T* Bs = As + ST_A;
    const R sg = tk.term[(kb + kt) / spt].neg ? (R)-1 : (R)1;
#pragma unroll 8
    for (int kk = 0; kk < BK; ++kk) {
      T a[TM], x[TN];
#pragma unroll
      for (int q = 0; q < TM; ++q) {
        a[q] = As[(ty * TM + q) * BK + kk];
        a[q].x *= sg;
        a[q].y *= sg;
      }
#pragma unroll
      for (int q = 0; q < TN; ++q) x[q] = Bs[kk * BN + tx * TN + q];
#pragma unroll
      for (int p = 0; p < TM; ++p)
#pragma unroll
        for (int q = 0; q < TN; ++q) {
          acc[p][q][0] = fma(a[p].x, x[q].x, acc[p][q][0]);
          acc[p][q][0] = fma(-a[p].y, x[q].y, acc[p][q][0]);
          acc[p][q][1] = fma(a[p].x, x[q].y, acc[p][q][1]);
          acc[p][q][1] = fma(a[p].y, x[q].x, acc[p][q][1]);
        }
    }
    __syncthreads();  // the slot is refilled by the issue of a later iteration
  }
  cp_async_wait<0>();
  T* out = reinterpret_cast<T*>(arrs.p[tk.out_arr]) + (size_t)tk.out_line * m * NC + (size_t)tk.s0 * C;
  const T* base = tk.base_arr ? reinterpret_cast<const T*>(arrs.p[tk.base_arr]) + (size_t)tk.base_line * m * NC +
                                    (size_t)tk.s0 * C
                              : nullptr;
#pragma unroll
  for (int p = 0; p < TM; ++p) {
    const int gr = row0 + ty * TM + p;
    if (gr >= m) continue;
#pragma unroll
    for (int q = 0; q < TN; ++q) {
      const int gc = col0 + tx * TN + q;
      if (gc >= ncols) continue;
      T z;
      z.x = acc[p][q][0];
      z.y = acc[p][q][1];
      if (partial) {
        partial[((size_t)blockIdx.z * m + gr) * totcols + s_coloff + gc] = z;
        continue;
      }
      T* o = out + (size_t)gr * NC + gc;
      const T b0 = base ? base[(size_t)gr * NC + gc] : (tk.mode == OUT_ADD ? *o : mk<T>(0, 0));
      *o = cadd(b0, z);
    }
  }
}

// Sum of the K slices of a grouped step in a fixed order, then each task's output rule.
// grid = (blocks over m * ns * C, ntask).
template <typename R>
__global__ void group_reduce_kernel(const typename Cx<R>::T* __restrict__ partial, int nsplit, int m,
                                    const GTask* __restrict__ tasks, GArrays arrs, int N, int C, int totcols) {
  using T = typename Cx<R>::T;
  const GTask& tk = tasks[blockIdx.y];
  int coloff = 0;
  for (int t = 0; t < (int)blockIdx.y; ++t) coloff += tasks[t].ns * C;
  const int ncols = tk.ns * C, NC = N * C;
  T* out = reinterpret_cast<T*>(arrs.p[tk.out_arr]) + (size_t)tk.out_line * m * NC + (size_t)tk.s0 * C;
  const T* base = tk.base_arr ? reinterpret_cast<const T*>(arrs.p[tk.base_arr]) + (size_t)tk.base_line * m * NC +
                                    (size_t)tk.s0 * C
                              : nullptr;
  const size_t total = (size_t)m * ncols, slice = (size_t)m * totcols;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
    const int gr = (int)(idx / ncols), gc = (int)(idx % ncols);
    const size_t pi = (size_t)gr * totcols + coloff + gc;
    T z = partial[pi];
    for (int k = 1; k < nsplit; ++k) z = cadd(z, partial[(size_t)k * slice + pi]);
    T* o = out + (size_t)gr * NC + gc;
    const T b0 = base ? base[(size_t)gr * NC + gc] : (tk.mode == OUT_ADD ? *o : mk<T>(0, 0));
    *o = cadd(b0, z);
  }
}

// Copy of one line, strips s0 .. s0+ns-1 (task 0 of a PH_COPY phase: term 0 -> output line).
template <typename T>
__global__ void copy_line_kernel(const T* __restrict__ src, T* __restrict__ dst, int m, int NC, int off, int cols) {
  const size_t total = (size_t)m * cols;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
    const size_t e = (idx / cols) * NC + off + idx % cols;
    dst[e] = src[e];
  }
}

// ------------------------------------------------------------------ tensor-core form
// One 3-D view per sweep array (floats of a node row, node rows, lines), box 2 BNC floats x
// 16 rows x 1 line: the raw input rows of a stage.
struct GMaps {
  CUtensorMap m[SB_COUNT];  // 16-row boxes: plain input rows, base rows
  CUtensorMap s[SB_COUNT];  // 18-row boxes: line-coupled input rows (one halo row each side)
};

// grid = (ceil(m / 128), total column tiles of the tasks (BNC columns each), nsplit), 320
// threads, the roles of tc_line_gemm_kernel: lane 0 of warp 8 issues the TMA loads (factor
// tiles hi and lo of term q's block; the raw rows of term q's input: 16 rows of a plain line,
// or 18 rows of a line-coupled one with a halo row each side, after the term's 16 base rows
// if it has a base), lane 0 of warp 9 the MMAs (TF32 x 3 into one FP32 accumulator in tensor
// memory), warps 0-7 build the B tiles (x = base +- C(input), split hi + lo, swizzled) and run
// the epilogue.  The coupling C to the node line below / above takes vert (vedge at the line's
// end nodes, vint inside) times the node plus dg times its neighbour along the line, as in the
// block-Thomas step.  K split z covers stages [z kst, (z+1) kst) of the concatenated terms.
// CLUSTER: the nsplit CTAs of a tile form a cluster (1, 1, nsplit) and sum their tiles in rank
// order through distributed shared memory.
template <class CF, bool CLUSTER>
__global__ void __launch_bounds__(tc::THREADS, 1)
    tc_group_kernel(const __grid_constant__ CUtensorMap map_hi, const __grid_constant__ CUtensorMap map_lo,
                    const __grid_constant__ GMaps maps, const GTask* __restrict__ tasks, int ntask, GArrays arrs,
                    int m, int N, int C, int kst, int split, float2 vedge, float2 vint, float dg, int* err,
                    long long budget) {
  using namespace tc;
  constexpr int BNC = CF::BNC, STAGES = CF::STAGES, BTILE = CF::BTILE;
  constexpr int STAGE_BYTES = CF::STAGE_BYTES, PAIR_GROUPS = CF::PAIR_GROUPS;
  constexpr int PAIRS_PER_THREAD = CF::PAIRS_PER_THREAD, TMEM_COLS = CF::TMEM_COLS, RAW_ROW = CF::RAW_ROW;
  extern __shared__ __align__(1024) unsigned char tc_smem_raw[];
  const uint32_t raw_s = smem_u32(tc_smem_raw);
  unsigned char* sm = tc_smem_raw + ((1024u - (raw_s & 1023u)) & 1023u);
  uint64_t* full_a = reinterpret_cast<uint64_t*>(sm + STAGES * STAGE_BYTES);
  uint64_t* full_b = full_a + STAGES;
  uint64_t* empty = full_b + STAGES;
  uint64_t* accfull = empty + STAGES;
  uint32_t* taddr_s = reinterpret_cast<uint32_t*>(accfull + 1);
  int* abort_s = reinterpret_cast<int*>(taddr_s + 1);
  __shared__ GTask tk;
  __shared__ int s_tile;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    int by = blockIdx.y, ti = 0;
    for (; ti < ntask - 1; ++ti) {
      const int tiles = (tasks[ti].ns * C + BNC - 1) / BNC;
      if (by < tiles) break;
      by -= tiles;
    }
    tk = tasks[ti];
    s_tile = by;
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full_a[s], 1);
      mbar_init(&full_b[s], BUILDERS);
      mbar_init(&empty[s], 1);
    }
    mbar_init(accfull, 1);
    *abort_s = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    fence_proxy_async();
  }
  if (warp == TMA_WARP) {
    tc::tmem_alloc(taddr_s, TMEM_COLS);
    tc::tmem_relinquish();
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = *taddr_s;
  const int row0 = blockIdx.x * BM;
  const int colc0 = s_tile * BNC;
  const int ncols = tk.ns * C;
  const int spt = (m + BKC - 1) / BKC, nst = tk.nterm * spt;
  const int kb = blockIdx.z * kst, ke = min(nst, kb + kst);
  const int nk = ke > kb ? ke - kb : 0;

  if (warp == TMA_WARP) {
    // ---------------------------------------------------------------- TMA issuer
    if (lane == 0) {
      auto load_a = [&](int kt) {
        const int s = kt % STAGES, st = kb + kt;
        const int q = st / spt, k0 = (st % spt) * BKC;
        const GTerm& g = tk.term[q];
        const int raw = (g.barr ? RAW_BASE_ROWS * RAW_ROW : 0) + (g.cpl ? RAW_SRC_ROWS : RAW_BASE_ROWS) * RAW_ROW;
        unsigned char* stp = sm + (size_t)s * STAGE_BYTES;
        if (split) {
          // map_hi is the complex64 store itself: the builders split the tile into hi + lo
          mbar_expect_tx(&full_a[s], TILE + raw);
          tc::tma_load_3d(stp, &map_hi, 2 * k0, row0, g.f, &full_a[s]);
        } else {
          mbar_expect_tx(&full_a[s], 2 * TILE + raw);
          tc::tma_load_3d(stp, &map_hi, 2 * k0, row0, g.f, &full_a[s]);
          tc::tma_load_3d(stp + TILE, &map_lo, 2 * k0, row0, g.f, &full_a[s]);
        }
      };
      auto load_raw = [&](int kt) {
        const int s = kt % STAGES, st = kb + kt;
        const int q = st / spt, k0 = (st % spt) * BKC;
        const GTerm& g = tk.term[q];
        unsigned char* rawp = sm + (size_t)s * STAGE_BYTES + 2 * TILE;
        // float index of the tile's first column in the input rows: even C keeps it a multiple
        // of 4 floats (16 bytes); strips outside 0..N-1 read the zero fill, and so do the halo
        // rows before node 0 and after node m-1
        if (g.barr) tc::tma_load_3d(rawp, &maps.m[g.barr], 2 * (tk.s0 * C + colc0), k0, g.bline, &full_a[s]);
        const int xs = 2 * ((tk.s0 + g.ds) * C + colc0);
        if (g.cpl)
          tc::tma_load_3d(rawp + RAW_BASE_ROWS * RAW_ROW, &maps.s[g.arr], xs, k0 - 1, g.line, &full_a[s]);
        else
          tc::tma_load_3d(rawp + RAW_BASE_ROWS * RAW_ROW, &maps.m[g.arr], xs, k0, g.line, &full_a[s]);
      };
      const int pre = min(nk, STAGES);
      for (int kt = 0; kt < pre; ++kt) load_a(kt);
      tc::griddep_wait();
      for (int kt = 0; kt < pre; ++kt) load_raw(kt);
      int issued = pre;
      for (int kt = pre; kt < nk; ++kt) {
        const int s = kt % STAGES;
        const unsigned ph = (unsigned)(kt / STAGES) & 1u;
        if (!mbar_wait(&empty[s], ph ^ 1u, err, budget)) { *(volatile int*)abort_s = 1; break; }
        if (tc::aborted(abort_s)) break;
        load_a(kt);
        load_raw(kt);
        issued = kt + 1;
      }
      if (tc::aborted(abort_s)) {
        for (int kt = max(0, issued - STAGES); kt < issued; ++kt)
          mbar_wait(&full_a[kt % STAGES], (unsigned)(kt / STAGES) & 1u, err, budget);
      }
    }
  } else if (warp == MMA_WARP) {
    // ---------------------------------------------------------------- MMA issuer
    if (lane == 0) {
      for (int kt = 0; kt < nk; ++kt) {
        const int s = kt % STAGES;
        const unsigned ph = (unsigned)(kt / STAGES) & 1u;
        if (!mbar_wait(&full_a[s], ph, err, budget) || !mbar_wait(&full_b[s], ph, err, budget)) {
          *(volatile int*)abort_s = 1;
          break;
        }
        if (tc::aborted(abort_s)) break;
        tc::fence_after();
        const uint32_t a_hi = smem_u32(sm + (size_t)s * STAGE_BYTES);
        const uint32_t a_lo = a_hi + TILE, b_hi = a_hi + 2 * TILE, b_lo = b_hi + BTILE;
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
          const uint32_t off = kk * 32;
          tc::mma_tf32(tmem, tc::sw128_desc(a_hi + off), tc::sw128_desc(b_hi + off), CF::IDESC, (kt | kk) != 0);
          tc::mma_tf32(tmem, tc::sw128_desc(a_hi + off), tc::sw128_desc(b_lo + off), CF::IDESC, 1);
          tc::mma_tf32(tmem, tc::sw128_desc(a_lo + off), tc::sw128_desc(b_hi + off), CF::IDESC, 1);
        }
        tc::commit(&empty[s]);
      }
      tc::commit(accfull);
      tc::griddep_launch_dependents();
    }
  } else {
    // ---------------------------------------------------------------- B builders
    const int c = threadIdx.x % BNC;
    const int pg = threadIdx.x / BNC;
    const bool cvalid = colc0 + c < ncols;
    for (int kt = 0; kt < nk; ++kt) {
      const int s = kt % STAGES;
      const unsigned ph = (unsigned)(kt / STAGES) & 1u;
      const int bad = (!mbar_wait(&full_a[s], ph, err, budget) || tc::aborted(abort_s)) ? 1 : 0;
      int any_bad;
      asm volatile(
          "{\n .reg .pred p, q;\n setp.ne.u32 q, %1, 0;\n bar.red.or.pred p, 1, %2, q;\n"
          " selp.u32 %0, 1, 0, p;\n}\n"
          : "=r"(any_bad)
          : "r"(bad), "n"(BUILDERS)
          : "memory");
      if (any_bad) {
        *(volatile int*)abort_s = 1;
        break;
      }
      const int st = kb + kt;
      const int k0 = (st % spt) * BKC;
      const GTerm& g = tk.term[st / spt];
      const float sg = g.neg ? -1.f : 1.f;
      if (split) {
        // A = hi + lo elementwise, the swizzled layout kept: hi in place, lo in the second tile
        float4* ah = reinterpret_cast<float4*>(sm + (size_t)s * STAGE_BYTES);
        float4* al = reinterpret_cast<float4*>(sm + (size_t)s * STAGE_BYTES + TILE);
        for (int e = threadIdx.x; e < TILE / 16; e += BUILDERS) {
          const float4 v = ah[e];
          float4 hv, lv;
          tc::split_tf32(v.x, hv.x, lv.x); tc::split_tf32(v.y, hv.y, lv.y);
          tc::split_tf32(v.z, hv.z, lv.z); tc::split_tf32(v.w, hv.w, lv.w);
          ah[e] = hv;
          al[e] = lv;
        }
      }
      unsigned char* bh = sm + (size_t)s * STAGE_BYTES + 2 * TILE;
      unsigned char* bl = bh + BTILE;
      const float2* rb = reinterpret_cast<const float2*>(bh);
      const float2* rs = reinterpret_cast<const float2*>(bh + RAW_BASE_ROWS * RAW_ROW);
      float2 x[2 * PAIRS_PER_THREAD];
#pragma unroll
      for (int u = 0; u < 2 * PAIRS_PER_THREAD; ++u) {
        const int kk = 2 * (pg + PAIR_GROUPS * (u >> 1)) + (u & 1);
        const int k = k0 + kk;
        float2 v = g.barr ? rb[kk * BNC + c] : make_float2(0.f, 0.f);
        float2 cp;
        if (g.cpl) {
          // raw row kk + 1 is node k; its neighbour along the line is row kk or kk + 2
          cp = rs[(kk + 1) * BNC + c];
          const int nb = g.cpl == XC_LOWER ? k - 1 : k + 1;
          const float2 y = (nb >= 0 && nb < m) ? rs[(kk + 1 + (g.cpl == XC_LOWER ? -1 : 1)) * BNC + c]
                                               : make_float2(0.f, 0.f);
          cp = cmul((k == 0 || k == m - 1) ? vedge : vint, cp);
          cp.x += dg * y.x;
          cp.y += dg * y.y;
        } else {
          cp = rs[kk * BNC + c];
        }
        v.x += sg * cp.x;
        v.y += sg * cp.y;
        x[u] = (k < m && cvalid) ? v : make_float2(0.f, 0.f);
      }
      asm volatile("bar.sync 1, %0;" ::"n"(BUILDERS) : "memory");
#pragma unroll
      for (int q = 0; q < PAIRS_PER_THREAD; ++q) {
        const int j = pg + PAIR_GROUPS * q;
        const float2 x0 = x[2 * q], x1 = x[2 * q + 1];
        const float re4[4] = {x0.x, -x0.y, x1.x, -x1.y};
        const float im4[4] = {x0.y, x0.x, x1.y, x1.x};
        float4 rh, rl, ih, il;
        tc::split_tf32(re4[0], rh.x, rl.x); tc::split_tf32(re4[1], rh.y, rl.y);
        tc::split_tf32(re4[2], rh.z, rl.z); tc::split_tf32(re4[3], rh.w, rl.w);
        tc::split_tf32(im4[0], ih.x, il.x); tc::split_tf32(im4[1], ih.y, il.y);
        tc::split_tf32(im4[2], ih.z, il.z); tc::split_tf32(im4[3], ih.w, il.w);
        *reinterpret_cast<float4*>(bh + tc::sw128_off(c, j)) = rh;
        *reinterpret_cast<float4*>(bl + tc::sw128_off(c, j)) = rl;
        *reinterpret_cast<float4*>(bh + tc::sw128_off(BNC + c, j)) = ih;
        *reinterpret_cast<float4*>(bl + tc::sw128_off(BNC + c, j)) = il;
      }
      fence_proxy_async_smem();
      mbar_arrive(&full_b[s]);
    }

    // ---------------------------------------------------------------- epilogue
    __syncwarp();
    // (the commit of an empty K range arrives at once; it is still awaited, so that no arrival
    // is pending when the CTA leaves)
    const bool ok = mbar_wait(accfull, 0, err, budget) && nk > 0;
    __syncwarp();
    tc::griddep_wait();
    tc::fence_after();
    float2* stile = reinterpret_cast<float2*>(sm);
    constexpr int SROW = BNC + 2;
    for (int h = warp >> 2; h < BNC / 32; h += BUILDERS / 128) {
      const int wq = warp & 3;
      const int r = wq * 32 + lane;
      const uint32_t trow = tmem + ((uint32_t)(wq * 32) << 16);
      uint32_t re[32], im[32];
      tc::tmem_ld32(trow + 32 * h, re);
      tc::tmem_ld32(trow + BNC + 32 * h, im);
      tc::tmem_wait_ld();
#pragma unroll
      for (int q = 0; q < 32; q += 2)
        *reinterpret_cast<float4*>(stile + r * SROW + 32 * h + q) =
            ok ? make_float4(__uint_as_float(re[q]), __uint_as_float(im[q]), __uint_as_float(re[q + 1]),
                             __uint_as_float(im[q + 1]))
               : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    asm volatile("bar.sync 2, %0;" ::"n"(BUILDERS) : "memory");
    if (!CLUSTER && ok && !tc::aborted(abort_s)) {
      const int NC = N * C;
      float2* out = reinterpret_cast<float2*>(arrs.p[tk.out_arr]) + (size_t)tk.out_line * m * NC + (size_t)tk.s0 * C;
      const float2* base = tk.base_arr ? reinterpret_cast<const float2*>(arrs.p[tk.base_arr]) +
                                             (size_t)tk.base_line * m * NC + (size_t)tk.s0 * C
                                       : nullptr;
      for (int e = threadIdx.x; e < BM * (BNC / 2); e += BUILDERS) {
        const int r = e / (BNC / 2), l = e % (BNC / 2);
        const int gr = row0 + r, gc = colc0 + 2 * l;
        if (gr >= m || gc >= ncols) continue;
        const float4 v = *reinterpret_cast<const float4*>(stile + r * SROW + 2 * l);
        float2* o = out + (size_t)gr * NC + gc;
        const float2* b = base ? base + (size_t)gr * NC + gc : nullptr;
        const bool two = gc + 1 < ncols;
        float2 b0 = b ? b[0] : (tk.mode == OUT_ADD ? o[0] : make_float2(0.f, 0.f));
        o[0] = make_float2(b0.x + v.x, b0.y + v.y);
        if (two) {
          const float2 b1 = b ? b[1] : (tk.mode == OUT_ADD ? o[1] : make_float2(0.f, 0.f));
          o[1] = make_float2(b1.x + v.z, b1.y + v.w);
        }
      }
    }
  }
  tc::fence_before();
  __syncthreads();
  if constexpr (CLUSTER) {
    tc::griddep_wait();
    constexpr int SROW = BNC + 2;
    const float2* stile = reinterpret_cast<const float2*>(sm);
    const unsigned nsplit = gridDim.z, q = tc::cluster_rank();
    tc::cluster_sync();
    const int rows = (BM + (int)nsplit - 1) / (int)nsplit, r0 = (int)q * rows;
    const bool good = !tc::aborted(abort_s) && *(volatile int*)err == 0;
    const int NC = N * C;
    float2* out = reinterpret_cast<float2*>(arrs.p[tk.out_arr]) + (size_t)tk.out_line * m * NC + (size_t)tk.s0 * C;
    const float2* base = tk.base_arr ? reinterpret_cast<const float2*>(arrs.p[tk.base_arr]) +
                                           (size_t)tk.base_line * m * NC + (size_t)tk.s0 * C
                                     : nullptr;
    for (int e = threadIdx.x; e < rows * (BNC / 2); e += THREADS) {
      const int r = r0 + e / (BNC / 2), l = e % (BNC / 2);
      if (r >= BM) break;
      const int gr = row0 + r, gc = colc0 + 2 * l;
      const bool live = good && gr < m && gc < ncols, two = gc + 1 < ncols;
      float2* o = out + (size_t)gr * NC + gc;
      float2 b0 = make_float2(0.f, 0.f), b1 = b0;
      if (live) {
        const float2* b = base ? base + (size_t)gr * NC + gc : (tk.mode == OUT_ADD ? o : nullptr);
        if (b) { b0 = b[0]; if (two) b1 = b[1]; }
      }
      float4 p[8];
#pragma unroll
      for (int z = 0; z < 8; ++z)
        if (z < (int)nsplit) p[z] = tc::ld_cluster_f4(stile + r * SROW + 2 * l, (unsigned)z);
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int z = 0; z < 8; ++z)
        if (z < (int)nsplit) { v.x += p[z].x; v.y += p[z].y; v.z += p[z].z; v.w += p[z].w; }
      if (!live) continue;
      o[0] = make_float2(b0.x + v.x, b0.y + v.y);
      if (two) o[1] = make_float2(b1.x + v.z, b1.y + v.w);
    }
    tc::cluster_sync();
  }
  if (warp == TMA_WARP) {
    tc::fence_after();
    tc::tmem_dealloc(tmem, TMEM_COLS);
  }
}

// ------------------------------------------------------------------ launchers
static int total_tiles(const SweepPhase& ph, int C, int bn) {
  int t = 0;
  for (const GTask& g : ph.tasks) t += (g.ns * C + bn - 1) / bn;
  return t;
}
static int max_terms(const SweepPhase& ph) {
  int q = 1;
  for (const GTask& g : ph.tasks) q = std::max(q, g.nterm);
  return q;
}

// CUDA-core grouped step (complex64 or complex128); the K split fills about two CTAs per SM
// and is limited by the slice buffer.
template <typename R>
cudaError_t launch_group_simt(Engine& E, const SweepPhase& ph, const GArrays& arrs, int C, void* partial_buf,
                              size_t partial_bytes) {
  using T = typename Cx<R>::T;
  // line-coupled terms (the twisted strip solves) run on the tensor-core kernels only
  for (const GTask& g : ph.tasks)
    for (int q = 0; q < g.nterm; ++q)
      if (g.term[q].cpl || g.term[q].barr) return cudaErrorInvalidValue;
  constexpr int BM = 64, BN = 64, BK = 16, STG = 3;
  constexpr size_t smem = (size_t)STG * (BM * BK + BK * BN) * sizeof(T);
  auto fn = group_gemm_kernel<R, BM, BN, BK, 4, 4, STG>;
  cudaFuncSetAttribute((const void*)fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  const int ntask = (int)ph.tasks.size();
  const int gx = (E.m + BM - 1) / BM, gy = total_tiles(ph, C, BN);
  int totcols = 0;
  for (const GTask& g : ph.tasks) totcols += g.ns * C;
  const int nst = max_terms(ph) * ((E.m + BK - 1) / BK);
  int nsplit = std::max(1, std::min(8, (2 * E.num_sms + gx * gy - 1) / (gx * gy)));
  while (nsplit > 1 && (size_t)nsplit * E.m * totcols * sizeof(T) > partial_bytes) --nsplit;
  const int kst = (nst + nsplit - 1) / nsplit;
  nsplit = (nst + kst - 1) / kst;
  const GTask* tasks = E.prog_tasks + ph.dev_off;
  T* partial = nsplit > 1 ? reinterpret_cast<T*>(partial_buf) : nullptr;
  fn<<<dim3(gx, gy, nsplit), 256, smem, E.stream>>>(reinterpret_cast<const T*>(E.factors), (size_t)E.m * E.ldf, E.ldf,
                                                    E.m, tasks, ntask, arrs, E.N, C, kst, partial, totcols);
  E.count_launch();
  if (nsplit > 1) {
    const int per = (int)std::min<size_t>(64, ((size_t)E.m * C * E.N + 255) / 256);
    group_reduce_kernel<R><<<dim3(std::max(1, per), ntask), 256, 0, E.stream>>>(partial, nsplit, E.m, tasks, arrs, E.N,
                                                                                C, totcols);
    E.count_launch();
  }
  return cudaGetLastError();
}

// Clusters of nsplit CTAs of the grouped step with tile shape CF that the device holds at once
// (one CTA per SM; a cluster needs its CTAs within one GPC, so fewer SMs are usable as the
// cluster grows), queried once per shape and size.
template <class CF>
static int group_cluster_fit(Engine& E, int nsplit) {
  const int key = CF::BNC * 16 + nsplit;
  const auto it = E.group_clusters.find(key);
  if (it != E.group_clusters.end()) return it->second;
  int n = E.num_sms / nsplit;
  if (nsplit > 1) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(1, 1, nsplit);
    cfg.blockDim = dim3(tc::THREADS);
    cfg.dynamicSmemBytes = CF::SMEM;
    cudaLaunchAttribute a[1];
    a[0].id = cudaLaunchAttributeClusterDimension;
    a[0].val.clusterDim.x = 1;
    a[0].val.clusterDim.y = 1;
    a[0].val.clusterDim.z = nsplit;
    cfg.attrs = a;
    cfg.numAttrs = 1;
    int q = 0;
    if (cudaOccupancyMaxActiveClusters(&q, (const void*)tc_group_kernel<CF, true>, &cfg) == cudaSuccess && q > 0)
      n = q;
    else
      cudaGetLastError();
  }
  n = std::max(1, n);
  E.group_clusters[key] = n;
  return n;
}

// Tensor-core grouped step: tile shape CF, K split into at most 8 slices summed in a cluster;
// the split minimises waves x (stages per slice + a fixed prologue / epilogue cost of about 6
// stages), the waves counted against the clusters that fit at once (18 clusters of 8 do not
// fit in one wave on 152 SMs: a two-task step of 9 row tiles each took twice its time so).
template <class CF>
static cudaError_t launch_tc_group_shape(Engine& E, const SweepPhase& ph, const GArrays& arrs, int C) {
  GMaps maps;
  std::memset(&maps, 0, sizeof(maps));
  for (int b = SB_RIN; b < SB_COUNT; ++b) {
    if (!arrs.p[b]) continue;
    const int lines = (b == SB_T0 || b == SB_T1) ? 1 : E.R + 1;
    const Engine::LineMaps* lm = E.line_maps_for(arrs.p[b], C, CF::BNC, lines);
    if (!lm) return cudaErrorInvalidValue;
    maps.m[b] = lm->base;
    maps.s[b] = lm->src;
  }
  const int ntask = (int)ph.tasks.size();
  const int gx = (E.m + tc::BM - 1) / tc::BM, gy = total_tiles(ph, C, CF::BNC);
  const int nst = max_terms(ph) * ((E.m + tc::BKC - 1) / tc::BKC);
  int nsplit = 1;
  {
    double best = 1e30;
    for (int ns = 1; ns <= 8; ++ns) {
      const int k_ns = (nst + ns - 1) / ns;
      const int fit = group_cluster_fit<CF>(E, ns);
      const int waves = (gx * gy + fit - 1) / fit;
      const double cost = waves * (k_ns + 6.0);
      if (cost < best) {
        best = cost;
        nsplit = ns;
      }
    }
  }
  const int kst = (nst + nsplit - 1) / nsplit;
  nsplit = (nst + kst - 1) / kst;
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(gx, gy, nsplit);
  cfg.blockDim = dim3(tc::THREADS);
  cfg.dynamicSmemBytes = CF::SMEM;
  cfg.stream = E.stream;
  cudaLaunchAttribute attr[2];
  unsigned na = 0;
  if (nsplit > 1) {
    attr[na].id = cudaLaunchAttributeClusterDimension;
    attr[na].val.clusterDim.x = 1;
    attr[na].val.clusterDim.y = 1;
    attr[na].val.clusterDim.z = nsplit;
    ++na;
  }
  if (E.opts.overlap_steps) {
    attr[na].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[na].val.programmaticStreamSerializationAllowed = 1;
    ++na;
  }
  cfg.attrs = attr;
  cfg.numAttrs = na;
  const GTask* tasks = E.prog_tasks + ph.dev_off;
  // split = 1 would read the factor tiles from the complex64 store and split them into TF32
  // hi + lo in shared memory (half the factor bytes); measured slower at k = 400 (2.82 against
  // 2.69 ms per sweep): these steps are not bound by HBM, and the splitting delays the MMAs
  const int split = 0;
  const CUtensorMap& fa = split ? E.tmap_c : E.tmap_hi;
  cudaError_t ce;
  const float2 vedge = E.coef.vert_f[0], vint = E.coef.vert_f[E.coef.n > 1 ? 1 : 0];
  const float dg = E.coef.diag_f;
  if (nsplit > 1)
    ce = cudaLaunchKernelEx(&cfg, tc_group_kernel<CF, true>, fa, E.tmap_lo, maps, tasks, ntask, arrs, E.m, E.N,
                            C, kst, split, vedge, vint, dg, E.err, E.opts.timeout_cycles);
  else
    ce = cudaLaunchKernelEx(&cfg, tc_group_kernel<CF, false>, fa, E.tmap_lo, maps, tasks, ntask, arrs, E.m, E.N,
                            C, kst, split, vedge, vint, dg, E.err, E.opts.timeout_cycles);
  E.count_launch();
  return ce;
}

cudaError_t launch_tc_group(Engine& E, int shape, const SweepPhase& ph, const GArrays& arrs, int C) {
  // a task wider than one 64-column tile but within one 128-column tile: the 128-column shape
  // reads each of its factor tiles once instead of once per column tile
  // (a phase with many tasks: the one-shot corrections; the scans and the two-task steps of
  // the twisted strip solves have too few tiles to fill the SMs without a K split, where the
  // 128-column tile's MMAs, twice as long per stage, set the pace: 1.86 against 2.02 ms per
  // k = 400 sweep with the twisted strip solves)
  if (shape == 0 && E.opts.group_wide_tiles) {
    int wmin = 1 << 30, wmax = 0;
    for (const GTask& g : ph.tasks) {
      wmin = std::min(wmin, g.ns * C);
      wmax = std::max(wmax, g.ns * C);
    }
    const int row_tiles = (E.m + tc::BM - 1) / tc::BM;
    if (wmin > tc::Wide::BNC && wmax <= tc::Huge::BNC && 2 * row_tiles * (int)ph.tasks.size() >= E.num_sms)
      shape = 2;
    // every task within one 32-column tile (the last strip's corrections of the twisted strip
    // solves at one right-hand side): the narrow shape, half the MMA work of the wide one
    if (wmax <= tc::Narrow::BNC) shape = 1;
  }
  if (shape == 1) return launch_tc_group_shape<tc::Narrow>(E, ph, arrs, C);
  if (shape == 2) return launch_tc_group_shape<tc::Huge>(E, ph, arrs, C);
  return launch_tc_group_shape<tc::Wide>(E, ph, arrs, C);
}

void set_tc_group_attributes() {
  cudaFuncSetAttribute((const void*)tc_group_kernel<tc::Wide, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)tc::Wide::SMEM);
  cudaFuncSetAttribute((const void*)tc_group_kernel<tc::Wide, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)tc::Wide::SMEM);
  cudaFuncSetAttribute((const void*)tc_group_kernel<tc::Narrow, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)tc::Narrow::SMEM);
  cudaFuncSetAttribute((const void*)tc_group_kernel<tc::Narrow, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)tc::Narrow::SMEM);
  cudaFuncSetAttribute((const void*)tc_group_kernel<tc::Huge, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)tc::Huge::SMEM);
  cudaFuncSetAttribute((const void*)tc_group_kernel<tc::Huge, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)tc::Huge::SMEM);
}

template <typename R>
cudaError_t launch_copy_phase(Engine& E, const SweepPhase& ph, const GArrays& arrs, int C) {
  using T = typename Cx<R>::T;
  const GTask& g = ph.tasks[0];
  const size_t NC = (size_t)E.N * C;
  const T* src = reinterpret_cast<const T*>(arrs.p[g.term[0].arr]) + (size_t)g.term[0].line * E.m * NC;
  T* dst = reinterpret_cast<T*>(arrs.p[g.out_arr]) + (size_t)g.out_line * E.m * NC;
  copy_line_kernel<T><<<E.grid_for((size_t)E.m * g.ns * C), 256, 0, E.stream>>>(src, dst, E.m, (int)NC, g.s0 * C,
                                                                               g.ns * C);
  E.count_launch();
  return cudaGetLastError();
}

template cudaError_t launch_group_simt<float>(Engine&, const SweepPhase&, const GArrays&, int, void*, size_t);
template cudaError_t launch_group_simt<double>(Engine&, const SweepPhase&, const GArrays&, int, void*, size_t);
template cudaError_t launch_copy_phase<float>(Engine&, const SweepPhase&, const GArrays&, int);
template cudaError_t launch_copy_phase<double>(Engine&, const SweepPhase&, const GArrays&, int);

}  // namespace hh
