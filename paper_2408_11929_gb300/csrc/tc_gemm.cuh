// Tensor-core form of the wide sweep step for complex64 data (sm_100 family: tcgen05 + TMA).
//
// One step computes out (op) F x for a factor block F (m x m complex) and right-hand-side
// lines x formed on the fly (x = base +- C(src), see LineOperand).  The complex product is
// one real GEMM:
//   D[r][n'] = sum_k' A[r][k'] B[n'][k'],   A[r][2k] = Re F(r,k), A[r][2k+1] = Im F(r,k)
// (the interleaved complex row of F read as 2m floats), and for complex column c of the tile
//   B[c][2k] = Re x, B[c][2k+1] = -Im x        -> D[r][c]      = Re (F x)(r, c)
//   B[64+c][2k] = Im x, B[64+c][2k+1] = Re x   -> D[r][64 + c] = Im (F x)(r, c)
// Precision: the MMA reads TF32 (11 significant bits), so every operand is split into
// hi = TF32(v) and lo = v - hi and the product is taken as hi*hi + hi*lo + lo*hi with FP32
// accumulation in tensor memory (about 2^-21 relative per product, against 2^-24 for an FP32
// FMA).  F's split is stored at setup; x is split while the B tile is built.
//
// CTA: 320 threads.  Lane 0 of warp 12 issues, per stage, four TMA loads on one mbarrier:
// the A tiles (hi, lo) and the raw line rows the stage's x is formed from (16 rows of the
// base line, 18 rows of the coupled line with one halo row each side), the raw rows landing
// in the slot's B area.  Eight warps build every stage's B tiles together (two node pairs
// per thread, so that each scheduler has two warps of short chains): they read the raw rows
// from shared memory, synchronise on a named barrier, and overwrite the area with the hi and
// lo B tiles (128-byte swizzled, K-major).  Warp 8 also owns the tensor-memory allocation;
// lane 0 of warp 9 issues the MMAs.  Epilogue: the eight warps move the accumulator (one row
// per thread, two column halves) into a padded shared tile, then write whole rows with
// coalesced 16-byte stores.  Three tile shapes are compiled: 64 complex columns with three
// 64 KB stages, 32 columns with four 48 KB stages, and 128 columns (the factor block is read
// by one column tile only) with two 96 KB stages; the sweep's autotuner picks one per column
// count.  Every wait is
#pragma once
#include <cuda.h>

#include "common.cuh"
#include "gemm.cuh"

namespace hh {
namespace tc {

constexpr int BM = 128;          // rows of F per CTA = tensor-memory lanes
constexpr int BKC = 16;          // complex node indices per stage
constexpr int TILE = 128 * 128;  // bytes of one A tile: 128 rows x 128 B
constexpr int BUILDERS = 256;    // 8 warps: B tiles, then the epilogue
constexpr int TMA_WARP = BUILDERS / 32, MMA_WARP = TMA_WARP + 1;
constexpr int THREADS = BUILDERS + 64;
constexpr int RAW_BASE_ROWS = BKC, RAW_SRC_ROWS = BKC + 2;

// Tile shape: BNC complex columns per CTA (MMA N = 2 BNC), STAGES ring slots.  Three shapes
// are compiled and the autotuner of the sweep picks one per column count.
template <int BNC_, int STAGES_>
struct Cfg {
  static constexpr int BNC = BNC_;
  static constexpr int BN = 2 * BNC_;  // real-part rows then imaginary-part rows of B
  static constexpr int STAGES = STAGES_;
  static constexpr int BTILE = BN * 128;  // bytes of one B tile: BN rows x 128 B
  static constexpr int STAGE_BYTES = 2 * TILE + 2 * BTILE;  // A hi, A lo, B hi, B lo
  static constexpr int PAIR_GROUPS = BUILDERS / BNC;                // threads per tile column
  static constexpr int PAIRS_PER_THREAD = (BKC / 2) / PAIR_GROUPS;  // node pairs per thread per stage
  static constexpr int TMEM_COLS = BN < 32 ? 32 : BN;              // a power of two, at least 32
  static constexpr int RAW_ROW = BNC * 8;  // bytes of one raw node row of the tile (complex64)
  static constexpr size_t SMEM = (size_t)STAGES * STAGE_BYTES + 1024 + 256;
  // instruction descriptor of kind::tf32: D F32 (bits 4-5 = 1), A and B TF32 (bits 7-9 and
  // 10-12 = 2), both K-major (bits 15, 16 = 0), N >> 3 at bits 17-22, M >> 4 at bits 24-28
  static constexpr uint32_t IDESC =
      (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
  static_assert(PAIRS_PER_THREAD >= 1 && (BKC / 2) % PAIR_GROUPS == 0, "builder mapping");
  static_assert(BNC % 32 == 0, "the epilogue moves 32 columns per tensor-memory load");
  static_assert(SMEM <= 232448, "shared memory");
};
using Wide = Cfg<64, 3>;
using Narrow = Cfg<32, 4>;
using Huge = Cfg<128, 2>;  // every column of a 4-direction sweep of one right-hand side in one tile

// shared-memory matrix descriptor, K-major, 128-byte swizzle: start address >> 4 (bits
// 0-13), leading offset unused by swizzled K-major layouts (1), stride offset between 8-row
// groups 1024 B >> 4 (bits 32-45), version 1 (bits 46-47), swizzle mode 2 = 128 B (61-63)
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// byte offset of 16-byte chunk j of row r in a 128-row tile with 128-byte swizzle
__device__ __forceinline__ uint32_t sw128_off(int r, int j) {
  return (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((j ^ (r & 7)) << 4));
}

// Programmatic dependent launch: wait until the preceding grid has completed and its memory
// is visible (immediate when the launch did not allow overlap), and let the next grid start
// its prologue once every CTA of this one has passed this point.
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void griddep_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// arrives on bar once every MMA issued so far by this thread has completed
__device__ __forceinline__ void commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void mma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}
// 32 consecutive 32-bit columns of this thread's lane
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
        "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]),
        "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
        "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr)
      : "memory");
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// 3-D tiled TMA load (x = float index along the row, y = row, z = factor block)
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

// hi = v rounded to the nearest TF32 value (11 significant bits), lo = v - hi (exact)
__device__ __forceinline__ void split_tf32(float v, float& hi, float& lo) {
  hi = __uint_as_float((__float_as_uint(v) + 0x1000u) & 0xFFFFE000u);
  lo = v - hi;
}

__device__ __forceinline__ bool aborted(const int* flag) { return *(volatile const int*)flag != 0; }

// thread-block clusters: rank of this CTA, all threads of the cluster meet, and a 16-byte
// load from the shared memory of another CTA of the cluster (same offset in its window)
__device__ __forceinline__ unsigned cluster_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\nbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ float4 ld_cluster_f4(const void* local, unsigned rank) {
  unsigned remote;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(smem_u32(local)), "r"(rank));
  float4 v;
  // no memory clobber: the reads follow a cluster barrier and may be issued back to back
  asm volatile("ld.shared::cluster.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "r"(remote));
  return v;
}

}  // namespace tc

// grid = (ceil(m / 128), ceil(ncols / 64), nsplit); split z covers node indices
// [z * kchunk, min(m, (z + 1) * kchunk)), kchunk a multiple of 16.  map_base / map_src: 3-D
// views (floats of a node row, node rows, lines) of the step's base and coupled sweep arrays
// (box 128 x 16 x 1 and 128 x 18 x 1; unused when the step has no such operand).  The column
// count per strip C must be even (16-byte aligned rows).  With partial != nullptr the CTA
// writes its slice to partial[(z * m + row) * ncols + col] for split_reduce_kernel, else it
// applies the step's output modes itself.
// CLUSTER: the K slices of a tile run as one thread-block cluster (cluster dims (1, 1,
// gridDim.z)) and are summed through distributed shared memory at the end, in rank order,
// instead of through partial (which must then be nullptr).
template <class CF, bool CLUSTER = false>
__global__ void __launch_bounds__(tc::THREADS, 1)
    tc_line_gemm_kernel(const __grid_constant__ CUtensorMap map_hi, const __grid_constant__ CUtensorMap map_lo,
                        const __grid_constant__ CUtensorMap map_base, const __grid_constant__ CUtensorMap map_src,
                        int fblock, int m, LineOperand<float2> op, Coef cf, int kchunk, float2* __restrict__ partial,
                        int* err, long long budget) {
  using namespace tc;
  constexpr int BNC = CF::BNC, BN = CF::BN, STAGES = CF::STAGES, BTILE = CF::BTILE;
  constexpr int STAGE_BYTES = CF::STAGE_BYTES, PAIR_GROUPS = CF::PAIR_GROUPS;
  constexpr int PAIRS_PER_THREAD = CF::PAIRS_PER_THREAD, TMEM_COLS = CF::TMEM_COLS, RAW_ROW = CF::RAW_ROW;
  (void)BN;
  extern __shared__ __align__(1024) unsigned char tc_smem_raw[];
  const uint32_t raw_s = smem_u32(tc_smem_raw);
  unsigned char* sm = tc_smem_raw + ((1024u - (raw_s & 1023u)) & 1023u);
  uint64_t* full_a = reinterpret_cast<uint64_t*>(sm + STAGES * STAGE_BYTES);  // TMA bytes landed
  uint64_t* full_b = full_a + STAGES;                                         // B tile built (BUILDERS arrivals)
  uint64_t* empty = full_b + STAGES;                                          // MMAs done reading
  uint64_t* accfull = empty + STAGES;                                         // accumulator final
  uint32_t* taddr_s = reinterpret_cast<uint32_t*>(accfull + 1);
  int* abort_s = reinterpret_cast<int*>(taddr_s + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row0 = blockIdx.x * BM;
  const int colc0 = blockIdx.y * BNC;
  const int ncols = op.ns * op.C;
  const int kbeg = blockIdx.z * kchunk;
  const int kend = min(m, kbeg + kchunk);
  const int nk = kend > kbeg ? (kend - kbeg + BKC - 1) / BKC : 0;
  const bool has_base = op.base != nullptr, has_src = op.cpl != XC_NONE;
  const int raw_bytes = (has_base ? RAW_BASE_ROWS * RAW_ROW : 0) + (has_src ? RAW_SRC_ROWS * RAW_ROW : 0);

  if (threadIdx.x == 0) {
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

  if (warp == TMA_WARP) {
    // ---------------------------------------------------------------- TMA issuer
    if (lane == 0) {
      // float index of this tile's first column in the base / coupled node rows (even C:
      // a multiple of 4 floats, i.e. 16-byte aligned)
      const int xb = 2 * (op.s0 * op.C + colc0);
      const int xs = 2 * ((op.s0 + op.src_ds) * op.C + colc0);
      auto load_a = [&](int kt) {
        const int s = kt % STAGES;
        unsigned char* st = sm + (size_t)s * STAGE_BYTES;
        mbar_expect_tx(&full_a[s], 2 * TILE + raw_bytes);
        const int x = 2 * (kbeg + kt * BKC);  // a multiple of 32 floats: 128-byte aligned
        tc::tma_load_3d(st, &map_hi, x, row0, fblock, &full_a[s]);
        tc::tma_load_3d(st + TILE, &map_lo, x, row0, fblock, &full_a[s]);
      };
      auto load_raw = [&](int kt) {
        const int s = kt % STAGES;
        unsigned char* rawp = sm + (size_t)s * STAGE_BYTES + 2 * TILE;
        const int k0 = kbeg + kt * BKC;
        if (has_base) tc::tma_load_3d(rawp, &map_base, xb, k0, op.base_j, &full_a[s]);
        if (has_src)
          tc::tma_load_3d(rawp + RAW_BASE_ROWS * RAW_ROW, &map_src, xs, k0 - 1, op.src_j, &full_a[s]);
      };
      // the factor tiles of the first ring slots do not depend on the preceding step: they
      // are requested before waiting for it, the line rows after
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
        // let every copy still in flight land before the CTA leaves
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
        for (int kk = 0; kk < 4; ++kk) {  // K = 8 TF32 values (32 bytes) per MMA
          const uint32_t off = kk * 32;
          tc::mma_tf32(tmem, tc::sw128_desc(a_hi + off), tc::sw128_desc(b_hi + off), CF::IDESC, (kt | kk) != 0);
          tc::mma_tf32(tmem, tc::sw128_desc(a_hi + off), tc::sw128_desc(b_lo + off), CF::IDESC, 1);
          tc::mma_tf32(tmem, tc::sw128_desc(a_lo + off), tc::sw128_desc(b_hi + off), CF::IDESC, 1);
        }
        tc::commit(&empty[s]);
      }
      tc::commit(accfull);
      tc::griddep_launch_dependents();  // every MMA of this CTA is issued
    }
  } else {
    // ---------------------------------------------------------------- B builders
    const int c = threadIdx.x % BNC;  // complex column within the tile
    const int pg = threadIdx.x / BNC;  // this thread forms node pairs pg, pg + PAIR_GROUPS, ... of a stage
    const bool cvalid = colc0 + c < ncols;
    const float2 vert_edge = cf.vert_f[0], vert_int = cf.vert_f[cf.n > 1 ? 1 : 0];
    const float dg = cf.diag_f;
    for (int kt = 0; kt < nk; ++kt) {
      const int s = kt % STAGES;
      const unsigned ph = (unsigned)(kt / STAGES) & 1u;
      // the builders decide together (barrier with OR reduction), so that all of them run
      // the same iterations and meet at the named barrier below
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
      const int k0 = kbeg + kt * BKC;
      unsigned char* bh = sm + (size_t)s * STAGE_BYTES + 2 * TILE;
      unsigned char* bl = bh + BTILE;
      // raw rows from shared memory: base row k - k0, coupled row k - k0 + 1
      const float2* rb = reinterpret_cast<const float2*>(bh);
      const float2* rs = reinterpret_cast<const float2*>(bh + RAW_BASE_ROWS * RAW_ROW);
      float2 x[2 * PAIRS_PER_THREAD];
#pragma unroll
      for (int u = 0; u < 2 * PAIRS_PER_THREAD; ++u) {
        const int kk = 2 * (pg + PAIR_GROUPS * (u >> 1)) + (u & 1);  // node within the stage
        const int k = k0 + kk;
        float2 v = has_base ? rb[kk * BNC + c] : make_float2(0.f, 0.f);
        if (has_src) {
          float2 cp = rs[(kk + 1) * BNC + c];
          if (op.cpl != XC_IDENT) {
            const int nb = op.cpl == XC_LOWER ? k - 1 : k + 1;
            const float2 y = (nb >= 0 && nb < m) ? rs[(kk + 1 + (op.cpl == XC_LOWER ? -1 : 1)) * BNC + c]
                                                 : make_float2(0.f, 0.f);
            cp = cmul((k == 0 || k == m - 1) ? vert_edge : vert_int, cp);
            cp.x += dg * y.x;
            cp.y += dg * y.y;
          }
          v = op.neg ? make_float2(v.x - cp.x, v.y - cp.y) : make_float2(v.x + cp.x, v.y + cp.y);
        }
        // nodes of the next split, and columns beyond the step, contribute nothing
        x[u] = (k < kend && cvalid) ? v : make_float2(0.f, 0.f);
      }
      // every builder has read its raw rows before any of them is overwritten
      asm volatile("bar.sync 1, %0;" ::"n"(BUILDERS) : "memory");
#pragma unroll
      for (int q = 0; q < PAIRS_PER_THREAD; ++q) {
        const int j = pg + PAIR_GROUPS * q;  // 16-byte chunk = node pair within the stage
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
      fence_proxy_async_smem();  // the tensor core reads these through the async proxy
      mbar_arrive(&full_b[s]);
    }

    // ---------------------------------------------------------------- epilogue
    // every MMA has completed once accfull fires, so the stage area is free: the accumulator
    // goes to a padded [128][BNC + 2] complex tile, then out by whole rows
    __syncwarp();
    const bool ok = mbar_wait(accfull, 0, err, budget);
    __syncwarp();
    tc::griddep_wait();  // the preceding grid's writes are visible before this one's
    tc::fence_after();
    float2* stile = reinterpret_cast<float2*>(sm);
    constexpr int SROW = BNC + 2;  // row stride (complex) of the staging tile
    // warp w reads tensor-memory lane quarter w % 4 (the only one it may access), complex
    // columns [32 h, 32 h + 32) for h = w / 4, w / 4 + 2, ...
    for (int h = warp >> 2; h < BNC / 32; h += BUILDERS / 128) {
      const int wq = warp & 3;       // tensor-memory lane quarter of this warp
      const int r = wq * 32 + lane;  // accumulator row
      const uint32_t trow = tmem + ((uint32_t)(wq * 32) << 16);
      uint32_t re[32], im[32];
      tc::tmem_ld32(trow + 32 * h, re);
      tc::tmem_ld32(trow + BNC + 32 * h, im);
      tc::tmem_wait_ld();
#pragma unroll
      for (int q = 0; q < 32; q += 2)
        *reinterpret_cast<float4*>(stile + r * SROW + 32 * h + q) =
            make_float4(__uint_as_float(re[q]), __uint_as_float(im[q]), __uint_as_float(re[q + 1]),
                        __uint_as_float(im[q + 1]));
    }
    asm volatile("bar.sync 2, %0;" ::"n"(BUILDERS) : "memory");
    if (!CLUSTER && ok && !tc::aborted(abort_s)) {
      const int N = op.N, C = op.C;
      // consecutive threads take consecutive column pairs (2l, 2l + 1) of a row
      for (int e = threadIdx.x; e < BM * (BNC / 2); e += BUILDERS) {
        const int r = e / (BNC / 2), l = e % (BNC / 2);
        const int gr = row0 + r;
        const int gc = colc0 + 2 * l;
        if (gr >= m || gc >= ncols) continue;
        const float4 v = *reinterpret_cast<const float4*>(stile + r * SROW + 2 * l);
        const float2 z0 = make_float2(v.x, v.y), z1 = make_float2(v.z, v.w);
        if (partial) {
          float2* p = partial + ((size_t)blockIdx.z * m + gr) * ncols + gc;
          if (gc + 1 < ncols) *reinterpret_cast<float4*>(p) = v;
          else *p = z0;
          continue;
        }
        // a node row of the sweep layout holds (strip, column) pairs contiguously
        float2* o = op.out + ((size_t)(op.out_j * m + gr) * N + op.s0) * C + gc;
        float2* a2 = op.acc ? op.acc + ((size_t)(op.acc_j * m + gr) * N + op.s0) * C + gc : nullptr;
        apply_out(o, z0, op.out_mode);
        if (a2) apply_out(a2, op.out_mode == OUT_SET ? z0 : *o, op.acc_mode);
        if (gc + 1 < ncols) {
          apply_out(o + 1, z1, op.out_mode);
          if (a2) apply_out(a2 + 1, op.out_mode == OUT_SET ? z1 : o[1], op.acc_mode);
        }
      }
    }
  }
  tc::fence_before();
  __syncthreads();
  if constexpr (CLUSTER) {
    tc::griddep_wait();  // every thread below may write the step's output
    // every CTA's staged tile is complete; CTA q of the cluster sums rows
    // [q BM / nsplit, (q + 1) BM / nsplit) of all tiles in rank order and writes them
    constexpr int SROW = BNC + 2;
    const float2* stile = reinterpret_cast<const float2*>(sm);
    const unsigned nsplit = gridDim.z, q = tc::cluster_rank();
    tc::cluster_sync();
    const int rows = (BM + (int)nsplit - 1) / (int)nsplit, r0 = (int)q * rows;
    const bool good = !tc::aborted(abort_s) && *(volatile int*)err == 0;
    const int N = op.N, C = op.C;
    auto upd = [](float2 cur, float2 z, int mode) {
      return mode == OUT_SET ? z : (mode == OUT_SUB ? make_float2(cur.x - z.x, cur.y - z.y)
                                                     : make_float2(cur.x + z.x, cur.y + z.y));
    };
    for (int e = threadIdx.x; e < rows * (BNC / 2); e += THREADS) {
      const int r = r0 + e / (BNC / 2), l = e % (BNC / 2);
      if (r >= BM) break;
      const int gr = row0 + r, gc = colc0 + 2 * l;
      const bool live = good && gr < m && gc < ncols, two = gc + 1 < ncols;
      float2* o = op.out + ((size_t)(op.out_j * m + gr) * N + op.s0) * C + gc;
      float2* a2 = op.acc ? op.acc + ((size_t)(op.acc_j * m + gr) * N + op.s0) * C + gc : nullptr;
      // the current output values and all slices' partial sums are requested together, so
      // that their latencies overlap; the slices are summed in rank order
      float2 o0 = make_float2(0.f, 0.f), o1 = o0, c0 = o0, c1 = o0;
      if (live && op.out_mode != OUT_SET) { o0 = o[0]; if (two) o1 = o[1]; }
      if (live && a2) { c0 = a2[0]; if (two) c1 = a2[1]; }
      float4 p[8];
#pragma unroll
      for (int z = 0; z < 8; ++z)
        if (z < (int)nsplit) p[z] = tc::ld_cluster_f4(stile + r * SROW + 2 * l, (unsigned)z);
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int z = 0; z < 8; ++z)
        if (z < (int)nsplit) { v.x += p[z].x; v.y += p[z].y; v.z += p[z].z; v.w += p[z].w; }
      if (!live) continue;
      // the second target takes the updated output (= the sum itself for OUT_SET)
      const float2 n0 = upd(o0, make_float2(v.x, v.y), op.out_mode);
      o[0] = n0;
      if (a2) a2[0] = upd(c0, n0, op.acc_mode);
      if (two) {
        const float2 n1 = upd(o1, make_float2(v.z, v.w), op.out_mode);
        o[1] = n1;
        if (a2) a2[1] = upd(c1, n1, op.acc_mode);
      }
    }
    tc::cluster_sync();  // no CTA leaves while another still reads its tile
  }
  if (warp == TMA_WARP) {
    tc::fence_after();
    tc::tmem_dealloc(tmem, TMEM_COLS);
  }
}

}  // namespace hh
