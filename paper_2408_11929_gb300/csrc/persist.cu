// One persistent launch per sweep (complex64 with an even column count, tensor cores).
//
// A sweep program (sweep.cu: block-Thomas or cyclic-reduction strip solves, interface scans,
// one-step interior corrections) is a sequence of phases; every phase is a set of
// independent output lines ("tasks", GTask), each a K-concatenated sum of factor blocks times
// input lines.  tc_persist_kernel runs ALL phases of a sweep in one cooperative launch of one
// CTA per SM:
//   * every phase is cut into work items (task, 128-row tile, BNC-column tile, K slice); the
//     CTAs take work items round robin;
//   * warp 8 (lane 0) streams the factor tiles and input rows of the CTA's work items through
//     a ring of shared-memory stages with TMA, continuously from one work item to the next;
//     warps 0-7 turn the input rows into the B tiles (x = base + (-1)^neg C(src), split into
//     TF32 hi + lo, 128-byte swizzled); lane 0 of warp 9 issues tcgen05.mma (TF32 x 3) into
//     one of two accumulators in tensor memory, alternating, so that the epilogue warps 10-13
//     read work item i while the MMAs of item i+1 run;
//   * a phase whose tiles would not fill the SMs splits K: every slice writes its partial tile
//     to an L2-resident buffer, and after a grid barrier all threads of the grid sum the slices
//     in a fixed order and apply the tasks' output rules;
//   * a grid barrier (bounded wait) separates the phases: a phase's input lines are complete
//     when it starts.
// Every wait is bounded: on expiry the device error word is set, every role stops, the copies in
// flight land, the tensor memory is freed and the kernel returns.
#include <algorithm>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include <cudaTypedefs.h>

#include "common.cuh"
#include "engine.h"
#include "gemm.cuh"
#include "tc_gemm.cuh"

namespace hh {

struct PPhase {
  int kind;              // PH_GROUP or PH_COPY
  int task_off, ntask;   // tasks in the persistent task table
  int ntiles;            // tiles of all tasks (row tiles x column tiles)
  int nsplit, kst;       // K slices of every tile, stages per slice
  int totcols;           // columns of all tasks (layout of the split-K partial tiles)
};

struct PMaps {
  CUtensorMap b[SB_COUNT];  // 16-row boxes (plain input rows, base rows)
  CUtensorMap s[SB_COUNT];  // 18-row boxes (coupled input rows, one halo row each side)
};

namespace pt {
constexpr int BUILDERS = 256;
constexpr int TMA_WARP = 8, MMA_WARP = 9, EPI_WARP0 = 10, EPI = 128;
constexpr int THREADS = BUILDERS + 64 + EPI;
}  // namespace pt

// Decoded work item of a phase.
struct PWork {
  const GTask* t;
  int row0, colc0, ncols, coloff, slice, kb, nk, spt;
};

template <int BNC>
__device__ __forceinline__ PWork decode_work(const PPhase& P, const GTask* tasks, int w, int m, int C) {
  PWork o;
  const int gx = (m + tc::BM - 1) / tc::BM;
  o.slice = w % P.nsplit;
  int tile = w / P.nsplit;
  const int rt = tile % gx;
  int ct = tile / gx;
  int ti = 0, coloff = 0;
  for (; ti < P.ntask - 1; ++ti) {
    const int cols = tasks[P.task_off + ti].ns * C, tl = (cols + BNC - 1) / BNC;
    if (ct < tl) break;
    ct -= tl;
    coloff += cols;
  }
  o.t = tasks + P.task_off + ti;
  o.row0 = rt * tc::BM;
  o.colc0 = ct * BNC;
  o.ncols = o.t->ns * C;
  o.coloff = coloff;
  o.spt = (m + tc::BKC - 1) / tc::BKC;
  const int nst = o.t->nterm * o.spt;
  o.kb = o.slice * P.kst;
  const int ke = min(nst, o.kb + P.kst);
  o.nk = ke > o.kb ? ke - o.kb : 0;
  return o;
}

__device__ __forceinline__ void fence_proxy_async_global() { asm volatile("fence.proxy.async.global;" ::: "memory"); }

// SPLIT_IN_SMEM: the factor tiles come from the complex64 store and are split into TF32 hi + lo
// in shared memory by the builders (half the factor bytes); otherwise from the stored hi and lo
// parts (two TMA loads per stage, no splitting work)
template <class CF, bool SPLIT_IN_SMEM>
__global__ void __launch_bounds__(pt::THREADS, 1)
    tc_persist_kernel(const __grid_constant__ CUtensorMap map_c, const __grid_constant__ CUtensorMap map_hi,
                      const __grid_constant__ CUtensorMap map_lo, const __grid_constant__ PMaps maps, const PPhase* __restrict__ phases, int nphase,
                      const GTask* __restrict__ tasks, GArrays arrs, int m, int N, int C, Coef cf,
                      float2* __restrict__ partial, unsigned* bar, int* err, long long budget) {
  using namespace tc;
  constexpr int BNC = CF::BNC, STAGES = CF::STAGES, BTILE = CF::BTILE;
  constexpr int STAGE_BYTES = CF::STAGE_BYTES, PAIR_GROUPS = CF::PAIR_GROUPS;
  constexpr int PAIRS_PER_THREAD = CF::PAIRS_PER_THREAD, TMEM_COLS = CF::TMEM_COLS, RAW_ROW = CF::RAW_ROW;
  constexpr uint32_t TMEM_ALLOC = 2 * TMEM_COLS;  // two accumulators
  extern __shared__ __align__(1024) unsigned char tc_smem_raw[];
  const uint32_t raw_s = smem_u32(tc_smem_raw);
  unsigned char* sm = tc_smem_raw + ((1024u - (raw_s & 1023u)) & 1023u);
  uint64_t* full_a = reinterpret_cast<uint64_t*>(sm + STAGES * STAGE_BYTES);
  uint64_t* full_b = full_a + STAGES;
  uint64_t* empty = full_b + STAGES;
  uint64_t* accfull = empty + STAGES;   // [2]: accumulator b complete (MMA commit)
  uint64_t* accempty = accfull + 2;     // [2]: accumulator b read by the epilogue (128 arrivals)
  uint32_t* taddr_s = reinterpret_cast<uint32_t*>(accempty + 2);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full_a[s], 1);
      mbar_init(&full_b[s], pt::BUILDERS);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&accfull[b], 1);
      mbar_init(&accempty[b], pt::EPI);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    fence_proxy_async();
  }
  if (warp == pt::TMA_WARP) {
    tc::tmem_alloc(taddr_s, TMEM_ALLOC);
    tc::tmem_relinquish();
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = *taddr_s;
  const int NC = N * C;
  const float2 vert_edge = cf.vert_f[0], vert_int = cf.vert_f[cf.n > 1 ? 1 : 0];
  const float dg = cf.diag_f;

  // TMA issue of stage kt of work item W into ring slot s: the factor tile (with the stage's
  // whole transaction count), and the input rows
  auto issue_a = [&](const PWork& W, int kt, int s) {
    const int st = W.kb + kt, q = st / W.spt, k0 = (st % W.spt) * BKC;
    const GTerm& g = W.t->term[q];
    const int raw = (g.barr ? RAW_BASE_ROWS * RAW_ROW : 0) + (g.cpl ? RAW_SRC_ROWS : RAW_BASE_ROWS) * RAW_ROW;
    if (SPLIT_IN_SMEM) {
      // the factor tile as stored (complex64): the builders split it into TF32 hi + lo
      mbar_expect_tx(&full_a[s], TILE + raw);
      tc::tma_load_3d(sm + (size_t)s * STAGE_BYTES, &map_c, 2 * k0, W.row0, g.f, &full_a[s]);
    } else {
      // the stored TF32 hi and lo parts of the factor tile
      mbar_expect_tx(&full_a[s], 2 * TILE + raw);
      tc::tma_load_3d(sm + (size_t)s * STAGE_BYTES, &map_hi, 2 * k0, W.row0, g.f, &full_a[s]);
      tc::tma_load_3d(sm + (size_t)s * STAGE_BYTES + TILE, &map_lo, 2 * k0, W.row0, g.f, &full_a[s]);
    }
  };
  auto issue_rows = [&](const PWork& W, int kt, int s) {
    const int st = W.kb + kt, q = st / W.spt, k0 = (st % W.spt) * BKC;
    const GTerm& g = W.t->term[q];
    unsigned char* rawp = sm + (size_t)s * STAGE_BYTES + 2 * TILE;
    if (g.barr) tc::tma_load_3d(rawp, &maps.b[g.barr], 2 * (W.t->s0 * C + W.colc0), k0, g.bline, &full_a[s]);
    const int xs = 2 * ((W.t->s0 + g.ds) * C + W.colc0);
    if (g.cpl)
      tc::tma_load_3d(rawp + RAW_BASE_ROWS * RAW_ROW, &maps.s[g.arr], xs, k0 - 1, g.line, &full_a[s]);
    else
      tc::tma_load_3d(rawp + RAW_BASE_ROWS * RAW_ROW, &maps.b[g.arr], xs, k0, g.line, &full_a[s]);
  };
  uint32_t it = 0;   // ring stages this thread's role has passed (same sequence in every role)
  uint32_t ai = 0;   // work items this CTA has run (accumulator ai & 1)
  uint32_t issued_total = 0;  // TMA: stages issued
  int npre = 0, pre_phase = -1;  // TMA: factor tiles of the next phase's first stages requested early
  unsigned target = 0;
  bool dead = false;
  for (int p = 0; p < nphase && !dead; ++p) {
    const PPhase P = phases[p];
    if (P.kind == PH_GROUP) {
      const int nwork = P.ntiles * P.nsplit;
      if (warp == pt::TMA_WARP) {
        // ---------------------------------------------------------- TMA producer
        if (lane == 0) {
          fence_proxy_async_global();  // lines written by the previous phases (generic stores)
          for (int w = blockIdx.x; w < nwork && !dead; w += gridDim.x) {
            const PWork W = decode_work<BNC>(P, tasks, w, m, C);
            for (int kt = 0; kt < W.nk; ++kt) {
              const int s = it % STAGES;
              if (kt < npre && w == (int)blockIdx.x) {
                // its factor tile was requested before the grid barrier (see below)
              } else {
                if (!mbar_wait(&empty[s], ((it / STAGES) & 1u) ^ 1u, err, budget)) { dead = true; break; }
                issue_a(W, kt, s);
              }
              issue_rows(W, kt, s);
              ++it;
              ++issued_total;
            }
            if (*(volatile int*)err) dead = true;
          }
          npre = 0;
          // The factor tiles of the next phase's first stages do not depend on this phase's
          // outputs: request them now, so that they land while the grid meets at the barrier
          // (their input rows follow after it and complete the same transaction count).
          if (!dead && p + 1 < nphase) {
            const PPhase Q = phases[p + 1];
            if (Q.kind == PH_GROUP && (int)blockIdx.x < Q.ntiles * Q.nsplit) {
              const PWork W = decode_work<BNC>(Q, tasks, blockIdx.x, m, C);
              const int n = min(W.nk, STAGES);
              for (int kt = 0; kt < n; ++kt) {
                const uint32_t i2 = it + kt;
                const int s = i2 % STAGES;
                if (!mbar_wait(&empty[s], ((i2 / STAGES) & 1u) ^ 1u, err, budget)) { dead = true; break; }
                issue_a(W, kt, s);
                npre = kt + 1;
              }
              pre_phase = p + 1;
            }
          }
        }
      } else if (warp == pt::MMA_WARP) {
        // ---------------------------------------------------------- MMA issuer
        if (lane == 0) {
          for (int w = blockIdx.x; w < nwork && !dead; w += gridDim.x) {
            const PWork W = decode_work<BNC>(P, tasks, w, m, C);
            const uint32_t b = ai & 1u;
            if (!mbar_wait(&accempty[b], ((ai >> 1) & 1u) ^ 1u, err, budget)) { dead = true; break; }
            tc::fence_after();
            const uint32_t acc = tmem + b * TMEM_COLS;
            for (int kt = 0; kt < W.nk; ++kt) {
              const int s = it % STAGES;
              const unsigned ph = (it / STAGES) & 1u;
              if (!mbar_wait(&full_a[s], ph, err, budget) || !mbar_wait(&full_b[s], ph, err, budget)) {
                dead = true;
                break;
              }
              tc::fence_after();
              const uint32_t a_hi = smem_u32(sm + (size_t)s * STAGE_BYTES);
              const uint32_t a_lo = a_hi + TILE, b_hi = a_hi + 2 * TILE, b_lo = b_hi + BTILE;
#pragma unroll
              for (int kk = 0; kk < 4; ++kk) {
                const uint32_t off = kk * 32;
                tc::mma_tf32(acc, tc::sw128_desc(a_hi + off), tc::sw128_desc(b_hi + off), CF::IDESC, (kt | kk) != 0);
                tc::mma_tf32(acc, tc::sw128_desc(a_hi + off), tc::sw128_desc(b_lo + off), CF::IDESC, 1);
                tc::mma_tf32(acc, tc::sw128_desc(a_lo + off), tc::sw128_desc(b_hi + off), CF::IDESC, 1);
              }
              tc::commit(&empty[s]);
              ++it;
            }
            tc::commit(&accfull[b]);
            ++ai;
            if (*(volatile int*)err) dead = true;
          }
        }
      } else if (warp < pt::TMA_WARP) {
        // ---------------------------------------------------------- B builders
        const int c = threadIdx.x % BNC;
        const int pg = threadIdx.x / BNC;
        for (int w = blockIdx.x; w < nwork && !dead; w += gridDim.x) {
          const PWork W = decode_work<BNC>(P, tasks, w, m, C);
          const bool cvalid = W.colc0 + c < W.ncols;
          for (int kt = 0; kt < W.nk; ++kt) {
            const int s = it % STAGES;
            const unsigned ph = (it / STAGES) & 1u;
            const int bad = (!mbar_wait(&full_a[s], ph, err, budget) || *(volatile int*)err) ? 1 : 0;
            int any_bad;
            asm volatile(
                "{\n .reg .pred p, q;\n setp.ne.u32 q, %1, 0;\n bar.red.or.pred p, 1, %2, q;\n"
                " selp.u32 %0, 1, 0, p;\n}\n"
                : "=r"(any_bad)
                : "r"(bad), "n"(pt::BUILDERS)
                : "memory");
            if (any_bad) { dead = true; break; }
            const int st = W.kb + kt, q = st / W.spt, k0 = (st % W.spt) * BKC;
            const GTerm& g = W.t->term[q];
            if (SPLIT_IN_SMEM) {
              // A = hi + lo elementwise (the swizzled layout is kept): hi in place, lo in the
              // second tile
              float4* ah = reinterpret_cast<float4*>(sm + (size_t)s * STAGE_BYTES);
              float4* al = reinterpret_cast<float4*>(sm + (size_t)s * STAGE_BYTES + TILE);
#pragma unroll
              for (int e = threadIdx.x; e < TILE / 16; e += pt::BUILDERS) {
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
            const float sg = g.neg ? -1.f : 1.f;
            float2 x[2 * PAIRS_PER_THREAD];
#pragma unroll
            for (int u = 0; u < 2 * PAIRS_PER_THREAD; ++u) {
              const int kk = 2 * (pg + PAIR_GROUPS * (u >> 1)) + (u & 1);
              const int k = k0 + kk;
              float2 v = g.barr ? rb[kk * BNC + c] : make_float2(0.f, 0.f);
              float2 cp;
              if (g.cpl) {
                cp = rs[(kk + 1) * BNC + c];
                const int nb = g.cpl == XC_LOWER ? k - 1 : k + 1;
                const float2 y = (nb >= 0 && nb < m) ? rs[(kk + 1 + (g.cpl == XC_LOWER ? -1 : 1)) * BNC + c]
                                                     : make_float2(0.f, 0.f);
                cp = cmul((k == 0 || k == m - 1) ? vert_edge : vert_int, cp);
                cp.x += dg * y.x;
                cp.y += dg * y.y;
              } else {
                cp = rs[kk * BNC + c];
              }
              v.x += sg * cp.x;
              v.y += sg * cp.y;
              x[u] = (k < m && cvalid) ? v : make_float2(0.f, 0.f);
            }
            asm volatile("bar.sync 1, %0;" ::"n"(pt::BUILDERS) : "memory");
#pragma unroll
            for (int qq = 0; qq < PAIRS_PER_THREAD; ++qq) {
              const int j = pg + PAIR_GROUPS * qq;
              const float2 x0 = x[2 * qq], x1 = x[2 * qq + 1];
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
            ++it;
          }
        }
      } else {
        // ---------------------------------------------------------- epilogue (warps 10-13)
        const int wq = warp & 3;          // tensor-memory lane quarter this warp may read
        const int r = wq * 32 + lane;     // accumulator row of this thread
        for (int w = blockIdx.x; w < nwork && !dead; w += gridDim.x) {
          const PWork W = decode_work<BNC>(P, tasks, w, m, C);
          const uint32_t b = ai & 1u;
          const bool ok = mbar_wait(&accfull[b], (ai >> 1) & 1u, err, budget);
          tc::fence_after();
          const int gr = W.row0 + r;
          const GTask& t = *W.t;
          float2* out = reinterpret_cast<float2*>(arrs.p[t.out_arr]) + (size_t)t.out_line * m * NC + (size_t)t.s0 * C;
          const float2* base = t.base_arr ? reinterpret_cast<const float2*>(arrs.p[t.base_arr]) +
                                                (size_t)t.base_line * m * NC + (size_t)t.s0 * C
                                          : nullptr;
          const uint32_t trow = tmem + b * TMEM_COLS + ((uint32_t)(wq * 32) << 16);
#pragma unroll 1
          for (int h = 0; h < BNC / 32; ++h) {
            uint32_t re[32], im[32];
            tc::tmem_ld32(trow + 32 * h, re);
            tc::tmem_ld32(trow + BNC + 32 * h, im);
            tc::tmem_wait_ld();
            if (!ok || gr >= m) continue;
            const int gc0 = W.colc0 + 32 * h;
            const float zf = W.nk ? 1.f : 0.f;  // an empty K slice contributes zero
            // 16-byte stores of column pairs (C even: the pairs never straddle the row end)
            if (P.nsplit > 1) {
              float4* pp = reinterpret_cast<float4*>(partial + ((size_t)W.slice * m + gr) * P.totcols + W.coloff + gc0);
#pragma unroll
              for (int q = 0; q < 32; q += 2)
                if (gc0 + q < W.ncols)
                  pp[q / 2] = make_float4(zf * __uint_as_float(re[q]), zf * __uint_as_float(im[q]),
                                          zf * __uint_as_float(re[q + 1]), zf * __uint_as_float(im[q + 1]));
            } else {
              float4* o = reinterpret_cast<float4*>(out + (size_t)gr * NC + gc0);
              const float4* bp = base ? reinterpret_cast<const float4*>(base + (size_t)gr * NC + gc0) : nullptr;
              float4 bv[16];
#pragma unroll
              for (int q = 0; q < 16; ++q)
                bv[q] = (gc0 + 2 * q < W.ncols && (bp || t.mode == OUT_ADD)) ? __ldcg(bp ? bp + q : o + q)
                                                                            : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
              for (int q = 0; q < 16; ++q)
                if (gc0 + 2 * q < W.ncols)
                  o[q] = make_float4(bv[q].x + zf * __uint_as_float(re[2 * q]), bv[q].y + zf * __uint_as_float(im[2 * q]),
                                     bv[q].z + zf * __uint_as_float(re[2 * q + 1]),
                                     bv[q].w + zf * __uint_as_float(im[2 * q + 1]));
            }
          }
          tc::fence_before();
          mbar_arrive(&accempty[b]);
          ++ai;
          if (!ok) dead = true;
        }
        fence_proxy_async_global();
      }
    } else if (P.kind == PH_COPY) {
      const GTask& t = tasks[P.task_off];
      const float2* src = reinterpret_cast<const float2*>(arrs.p[t.term[0].arr]) + (size_t)t.term[0].line * m * NC;
      float2* dst = reinterpret_cast<float2*>(arrs.p[t.out_arr]) + (size_t)t.out_line * m * NC;
      const size_t cols = (size_t)t.ns * C, total = (size_t)m * cols;
      for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
        const size_t e = (idx / cols) * NC + (size_t)t.s0 * C + idx % cols;
        dst[e] = __ldcg(src + e);
      }
      fence_proxy_async_global();
    }
    // every output line of the phase is in place before the next phase reads it
    if (!grid_sync(bar, target, err, budget)) { dead = true; break; }
    if (P.kind == PH_GROUP && P.nsplit > 1) {
      // the K slices of every tile, summed in slice order by all threads of the grid
      for (int ti = 0; ti < P.ntask; ++ti) {
        const GTask& t = tasks[P.task_off + ti];
        int coloff = 0;
        for (int u = 0; u < ti; ++u) coloff += tasks[P.task_off + u].ns * C;
        const int cols = t.ns * C;
        float2* out = reinterpret_cast<float2*>(arrs.p[t.out_arr]) + (size_t)t.out_line * m * NC + (size_t)t.s0 * C;
        const float2* base = t.base_arr ? reinterpret_cast<const float2*>(arrs.p[t.base_arr]) +
                                              (size_t)t.base_line * m * NC + (size_t)t.s0 * C
                                        : nullptr;
        const size_t total = (size_t)m * cols, slice = (size_t)m * P.totcols;
        // column pairs (C even), every slice's load in flight at once, summed in slice order
        const size_t pairs = total / 2;
        for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < pairs;
             idx += (size_t)gridDim.x * blockDim.x) {
          const int gr = (int)(2 * idx / cols), gc = (int)(2 * idx % cols);
          const size_t pi = (size_t)gr * P.totcols + coloff + gc;
          float4 pv[8];
#pragma unroll
          for (int k = 0; k < 8; ++k)
            if (k < P.nsplit) pv[k] = __ldcg(reinterpret_cast<const float4*>(partial + (size_t)k * slice + pi));
          float4* o = reinterpret_cast<float4*>(out + (size_t)gr * NC + gc);
          const float4 b0 = base ? __ldcg(reinterpret_cast<const float4*>(base + (size_t)gr * NC + gc))
                                 : (t.mode == OUT_ADD ? __ldcg(o) : make_float4(0.f, 0.f, 0.f, 0.f));
          float4 z = pv[0];
#pragma unroll
          for (int k = 1; k < 8; ++k)
            if (k < P.nsplit) { z.x += pv[k].x; z.y += pv[k].y; z.z += pv[k].z; z.w += pv[k].w; }
          *o = make_float4(b0.x + z.x, b0.y + z.y, b0.z + z.z, b0.w + z.w);
        }
      }
      fence_proxy_async_global();
      if (!grid_sync(bar, target, err, budget)) { dead = true; break; }
    }
  }
  // leave: copies in flight land (bounded), every thread done with tensor memory, free it
  if (warp == pt::TMA_WARP && lane == 0 && dead) {
    if (npre > 0 && pre_phase >= 0) {
      // early factor tiles whose input rows were never requested: request them, so that the
      // stages' transaction counts complete and the waits below see every copy land
      const PWork W = decode_work<BNC>(phases[pre_phase], tasks, blockIdx.x, m, C);
      for (int kt = 0; kt < npre; ++kt) {
        issue_rows(W, kt, (it + kt) % STAGES);
        ++issued_total;
      }
    }
    for (uint32_t q = issued_total > STAGES ? issued_total - STAGES : 0; q < issued_total; ++q)
      mbar_wait(&full_a[q % STAGES], (q / STAGES) & 1u, err, budget);
  }
  tc::fence_before();
  __syncthreads();
  if (warp == pt::TMA_WARP) {
    tc::fence_after();
    tc::tmem_dealloc(tmem, TMEM_ALLOC);
  }
}

// ------------------------------------------------------------------ host side
// A block-Thomas step of the line-coupled form (SweepStep) as a grouped task: x = base +-
// C(src), out (set / +=) F x.  A subtracting step negates x (its steps carry no base).
static bool step_to_task(const SweepStep& s, GTask& t) {
  if (s.acc != SB_NONE) return false;
  t = GTask{};
  t.nterm = 1;
  GTerm& g = t.term[0];
  g.f = s.f;
  if (s.src != SB_NONE && s.cpl != XC_NONE) {
    g.arr = s.src; g.line = s.src_j; g.ds = s.src_ds; g.neg = s.neg;
    g.cpl = s.cpl == XC_IDENT ? 0 : s.cpl;
    g.barr = s.base; g.bline = s.base_j;
  } else {
    g.arr = s.base; g.line = s.base_j; g.ds = 0; g.neg = 0; g.cpl = 0; g.barr = 0;
  }
  t.out_arr = s.out; t.out_line = s.out_j;
  t.base_arr = SB_NONE;
  t.mode = s.out_mode == OUT_SET ? OUT_SET : OUT_ADD;
  if (s.out_mode == OUT_SUB) {
    if (g.barr) return false;
    g.neg ^= 1;
  }
  t.s0 = s.s0; t.ns = s.ns;
  return true;
}

// The persistent programs of every stored depth (double and single sweep), as one device task
// table; phase lists on the host.  Returns false when a program has a step the kernel cannot
// run (it then stays on the per-phase launches).
int Engine::upload_persistent() {
  std::vector<GTask> all;
  for (int d = 0; d < NPROG; ++d)
    for (int single = 0; single < 2; ++single) {
      const std::vector<SweepPhase>& prog = single ? prog_single_d[d] : prog_double_d[d];
      std::vector<SweepPhase>& pp = single ? pprog_single_d[d] : pprog_double_d[d];
      pp.clear();
      bool ok = !prog.empty();
      for (const SweepPhase& ph : prog) {
        SweepPhase q;
        q.kind = ph.kind == PH_COPY ? PH_COPY : PH_GROUP;
        if (ph.kind == PH_STEP) {
          GTask t;
          if (!step_to_task(ph.step, t)) { ok = false; break; }
          q.tasks.push_back(t);
        } else {
          q.tasks = ph.tasks;
        }
        pp.push_back(q);
      }
      if (!ok) { pp.clear(); continue; }
      for (SweepPhase& ph : pp) {
        ph.dev_off = all.size();
        for (const GTask& t : ph.tasks) all.push_back(t);
      }
    }
  dfree(pprog_tasks);
  pprog_tasks = nullptr;
  if (all.empty()) return HH_OK;
  if (dmalloc((void**)&pprog_tasks, all.size() * sizeof(GTask))) return HH_ENOMEM;
  cudaMemcpy(pprog_tasks, all.data(), all.size() * sizeof(GTask), cudaMemcpyHostToDevice);
  return HH_OK;
}

template <class CF>
static int persist_smem() {
  return (int)((size_t)CF::STAGES * CF::STAGE_BYTES + 1024 + 256);
}

void set_persist_attributes() {
  cudaFuncSetAttribute((const void*)tc_persist_kernel<tc::Wide, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       persist_smem<tc::Wide>());
  cudaFuncSetAttribute((const void*)tc_persist_kernel<tc::Narrow, false>,
                       cudaFuncAttributeMaxDynamicSharedMemorySize, persist_smem<tc::Narrow>());
  cudaFuncSetAttribute((const void*)tc_persist_kernel<tc::Huge, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       persist_smem<tc::Huge>());
  cudaFuncSetAttribute((const void*)tc_persist_kernel<tc::Wide, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       persist_smem<tc::Wide>());
  cudaFuncSetAttribute((const void*)tc_persist_kernel<tc::Narrow, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       persist_smem<tc::Narrow>());
  cudaFuncSetAttribute((const void*)tc_persist_kernel<tc::Huge, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       persist_smem<tc::Huge>());
}

// Device phase table of a program for C columns and tile shape CF: tiles, K split, stages per
// slice.  Built (a host-to-device copy) outside stream capture; inside a capture only looked up.
template <class CF>
static PPhase* phase_table(Engine& E, const std::vector<SweepPhase>& prog, int C, size_t partial_bytes, int depth,
                           bool single) {
  const int64_t key = (((int64_t)depth * 2 + (single ? 1 : 0)) * 4 + (CF::BNC == 32 ? 1 : CF::BNC == 128 ? 2 : 0)) *
                          100000 + C;
  PPhase* dev = nullptr;
  const auto itc = E.pphase_cache.find(key);
  if (itc != E.pphase_cache.end()) return reinterpret_cast<PPhase*>(itc->second);
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(E.stream, &cs);
  if (cs != cudaStreamCaptureStatusNone) return nullptr;
  {
    std::vector<PPhase> ph;
    const int gx = (E.m + tc::BM - 1) / tc::BM, spt = (E.m + tc::BKC - 1) / tc::BKC;
    for (const SweepPhase& q : prog) {
      PPhase P{};
      P.kind = q.kind;
      P.task_off = (int)q.dev_off;
      P.ntask = (int)q.tasks.size();
      int tiles = 0, cols = 0, nterm = 1;
      for (const GTask& t : q.tasks) {
        tiles += (t.ns * C + CF::BNC - 1) / CF::BNC;
        cols += t.ns * C;
        nterm = std::max(nterm, t.nterm);
      }
      P.ntiles = tiles * gx;
      P.totcols = cols;
      int ns = 1;
      if (q.kind == PH_GROUP && P.ntiles < E.num_sms / 2) {
        ns = std::max(1, std::min(8, E.num_sms / std::max(1, P.ntiles)));
        while (ns > 1 && (size_t)ns * E.m * cols * sizeof(float2) > partial_bytes) --ns;
      }
      const int nst = nterm * spt;
      P.kst = (nst + ns - 1) / ns;
      P.nsplit = (nst + P.kst - 1) / P.kst;
      ph.push_back(P);
    }
    if (E.dmalloc((void**)&dev, ph.size() * sizeof(PPhase))) return nullptr;
    cudaMemcpy(dev, ph.data(), ph.size() * sizeof(PPhase), cudaMemcpyHostToDevice);
    E.pphase_cache[key] = dev;
  }
  return dev;
}

template <class CF>
static int run_persistent_shape(Engine& E, const std::vector<SweepPhase>& prog, const GArrays& arrs, int C,
                                void* partial_buf, size_t partial_bytes, int depth, bool single) {
  PPhase* dev = phase_table<CF>(E, prog, C, partial_bytes, depth, single);
  if (!dev) return HH_EINVAL;  // not prepared before a capture: the caller launches phase by phase
  PMaps maps;
  std::memset(&maps, 0, sizeof(maps));
  for (int b = SB_RIN; b < SB_COUNT; ++b) {
    if (!arrs.p[b]) continue;
    const int lines = (b == SB_T0 || b == SB_T1) ? 1 : E.R + 1;
    const Engine::LineMaps* lm = E.line_maps_for(arrs.p[b], C, CF::BNC, lines);
    if (!lm) return (set_error("tensor maps of the sweep arrays"), HH_ECUDA);
    maps.b[b] = lm->base;
    maps.s[b] = lm->src;
  }
  unsigned* pbar = E.bar + Engine::BAR_PERSIST * GRID_BAR_WORDS;
  cudaMemsetAsync(pbar, 0, GRID_BAR_WORDS * sizeof(unsigned), E.stream);
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(E.num_sms);
  cfg.blockDim = dim3(pt::THREADS);
  cfg.dynamicSmemBytes = persist_smem<CF>();
  cfg.stream = E.stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const int nphase = (int)prog.size();
  float2* partial = reinterpret_cast<float2*>(partial_buf);
  const cudaError_t ce =
      E.opts.persistent == 2
          ? cudaLaunchKernelEx(&cfg, tc_persist_kernel<CF, true>, E.tmap_c, E.tmap_hi, E.tmap_lo, maps,
                               (const PPhase*)dev, nphase, (const GTask*)E.pprog_tasks, arrs, E.m, E.N, C, E.coef,
                               partial, pbar, E.err, E.opts.timeout_cycles)
          : cudaLaunchKernelEx(&cfg, tc_persist_kernel<CF, false>, E.tmap_c, E.tmap_hi, E.tmap_lo, maps,
                               (const PPhase*)dev, nphase, (const GTask*)E.pprog_tasks, arrs, E.m, E.N, C, E.coef,
                               partial, pbar, E.err, E.opts.timeout_cycles);
  E.count_launch();
  if (ce != cudaSuccess) return (E.set_cuda_error(ce, "persistent sweep launch"), HH_ECUDA);
  return HH_OK;
}

// Builds the phase tables of the C-column programs (double and single sweep) for the chosen
// depth and tile shape; called before any stream capture of such a sweep.
int prepare_persistent(Engine& E, int C, size_t partial_bytes) {
  if (E.precision != HH_PREC_FP32 || !E.tc_ready || C % 2 || !E.opts.persistent || !E.pprog_tasks) return HH_OK;
  const int d = E.depth_for(C);
  const auto it = E.tc_tuned.find(C);
  const int shape = it != E.tc_tuned.end() ? it->second.shape : 0;
  for (int single = 0; single < 2; ++single) {
    const std::vector<SweepPhase>& prog = single ? E.pprog_single_d[d] : E.pprog_double_d[d];
    if (prog.empty()) continue;
    PPhase* dev = shape == 1 ? phase_table<tc::Narrow>(E, prog, C, partial_bytes, d, single != 0)
                             : shape == 2 ? phase_table<tc::Huge>(E, prog, C, partial_bytes, d, single != 0)
                                          : phase_table<tc::Wide>(E, prog, C, partial_bytes, d, single != 0);
    if (!dev) return HH_ENOMEM;
  }
  return HH_OK;
}

// One sweep as one persistent launch; HH_EINVAL when this sweep cannot run that way (the caller
// then launches phase by phase).
int run_persistent(Engine& E, const GArrays& arrs, int C, bool single, void* partial_buf, size_t partial_bytes) {
  if (E.precision != HH_PREC_FP32 || !E.tc_ready || C % 2 || !E.opts.persistent || !E.pprog_tasks) return HH_EINVAL;
  // the no-allocation entry point keeps to the phase launches (its slice buffer is the rest of
  // a fixed array, and a phase table may not be built during its call)
  if (E.no_alloc_call) return HH_EINVAL;
  const int d = E.depth_for(C);
  const std::vector<SweepPhase>& prog = single ? E.pprog_single_d[d] : E.pprog_double_d[d];
  if (prog.empty()) return HH_EINVAL;
  const auto it = E.tc_tuned.find(C);
  const int shape = it != E.tc_tuned.end() ? it->second.shape : 0;
  if (shape == 1) return run_persistent_shape<tc::Narrow>(E, prog, arrs, C, partial_buf, partial_bytes, d, single);
  if (shape == 2) return run_persistent_shape<tc::Huge>(E, prog, arrs, C, partial_buf, partial_bytes, d, single);
  return run_persistent_shape<tc::Wide>(E, prog, arrs, C, partial_buf, partial_bytes, d, single);
}

}  // namespace hh
