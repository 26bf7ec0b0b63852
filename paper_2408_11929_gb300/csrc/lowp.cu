// Lower-precision sweeps (hh_opts.precision = HH_PREC_BF16): the strip factors stored in
// bf16 and the sweep's products taken on the tensor cores as ONE tcgen05.mma.kind::f16 per K
// step with bf16 operands and FP32 accumulation (the complex64 path takes three TF32
// products per K step to reach FP32 accuracy).  The sweep lines stay complex64 and every step
// accumulates in FP32; only the factor entries and the line values entering a product are
// rounded to bf16 (8 significant bits).  Flexible GMRES takes the result as a different,
// fixed preconditioner: it still converges, and the cost shows as iterations (Section 5 of the
// paper names lower-precision subsolves as a way to cheaper sweeps).
//
// The sweep program is the one of the persistent kernel (every block-Thomas step as a grouped
// task with a line-coupled term, grouped steps, line copies), run phase by phase by
// tc_lowp_kernel: per stage 32 complex nodes (a 128-byte bf16 row), the factor tile by TMA
// (128 rows x 64 bf16, 128-byte swizzle), the input rows by TMA (32 base rows, 34 coupled
// rows with a halo row each side, or 32 plain rows), B built by 8 warps as bf16 (rows
// (Re x, -Im x) and (Im x, Re x) of every complex column), four MMAs of K = 16.  K split over
// a thread-block cluster, slices summed through distributed shared memory.
#include <algorithm>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include "common.cuh"
#include "engine.h"
#include "gemm.cuh"
#include "tc_gemm.cuh"

namespace hh {

template <typename R>
cudaError_t launch_copy_phase(Engine& E, const SweepPhase& ph, const GArrays& arrs, int C);

namespace lp {
constexpr int BKC = 32;                       // complex nodes per stage
constexpr int ATILE = 128 * 128;              // bytes of one bf16 factor tile (128 rows x 128 B)
constexpr int BASE_ROWS = BKC, SRC_ROWS = BKC + 2;

template <int BNC_, int STAGES_>
struct Cfg {
  static constexpr int BNC = BNC_;
  static constexpr int BN = 2 * BNC_;
  static constexpr int STAGES = STAGES_;
  static constexpr int BTILE = BN * 128;
  static constexpr int RAW_ROW = BNC * 8;
  static constexpr int RAW_BYTES = (BASE_ROWS + SRC_ROWS) * RAW_ROW;
  static constexpr int STAGE_BYTES = ((ATILE + BTILE + RAW_BYTES) + 1023) / 1024 * 1024;
  static constexpr int CHUNK_GROUPS = tc::BUILDERS / BNC;           // threads per complex column
  static constexpr int CHUNKS_PER_THREAD = 8 / CHUNK_GROUPS;        // 16-byte chunks of a row
  static constexpr int TMEM_COLS = BN < 32 ? 32 : BN;
  static constexpr size_t SMEM = (size_t)STAGES * STAGE_BYTES + 1024 + 256;
  // instruction descriptor of kind::f16: D F32 (bits 4-5 = 1), A and B BF16 (bits 7-9 and 10-12
  // = 1), both K-major, N >> 3 at bits 17-22, M >> 4 at bits 24-28
  static constexpr uint32_t IDESC =
      (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
  static_assert(CHUNKS_PER_THREAD >= 1 && 8 % CHUNK_GROUPS == 0, "builder mapping");
  static_assert(BNC % 32 == 0, "epilogue");
  static_assert(SMEM <= 232448, "shared memory");
};
using Wide = Cfg<64, 3>;
using Narrow = Cfg<32, 5>;

__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&v);
}
}  // namespace lp

// views of a sweep array with the input-row boxes of a bf16 stage (32 and 34 rows)
struct LMaps {
  CUtensorMap b[SB_COUNT];
  CUtensorMap s[SB_COUNT];
};

// grid = (ceil(m / 128), column tiles of all tasks, nsplit); CLUSTER: the nsplit CTAs of a tile
// are one cluster (1, 1, nsplit) and sum their tiles through distributed shared memory.
template <class CF, bool CLUSTER>
__global__ void __launch_bounds__(tc::THREADS, 1)
    tc_lowp_kernel(const __grid_constant__ CUtensorMap map_f, const __grid_constant__ LMaps maps,
                   const GTask* __restrict__ tasks, int ntask, GArrays arrs, int m, int N, int C, int kst, Coef cf,
                   int* err, long long budget) {
  using namespace tc;
  constexpr int BNC = CF::BNC, STAGES = CF::STAGES, BTILE = CF::BTILE, RAW_ROW = CF::RAW_ROW;
  constexpr int STAGE_BYTES = CF::STAGE_BYTES, CG = CF::CHUNK_GROUPS, CPT = CF::CHUNKS_PER_THREAD;
  constexpr int TMEM_COLS = CF::TMEM_COLS;
  extern __shared__ __align__(1024) unsigned char lp_smem_raw[];
  const uint32_t raw_s = smem_u32(lp_smem_raw);
  unsigned char* sm = lp_smem_raw + ((1024u - (raw_s & 1023u)) & 1023u);
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
  const int spt = (m + lp::BKC - 1) / lp::BKC, nst = tk.nterm * spt;
  const int kb = blockIdx.z * kst, ke = min(nst, kb + kst);
  const int nk = ke > kb ? ke - kb : 0;

  if (warp == TMA_WARP) {
    // ---------------------------------------------------------------- TMA issuer
    if (lane == 0) {
      auto load_a = [&](int kt) {
        const int s = kt % STAGES, st = kb + kt;
        const int q = st / spt, k0 = (st % spt) * lp::BKC;
        const GTerm& g = tk.term[q];
        const int raw = (g.barr ? lp::BASE_ROWS * RAW_ROW : 0) + (g.cpl ? lp::SRC_ROWS : lp::BASE_ROWS) * RAW_ROW;
        mbar_expect_tx(&full_a[s], lp::ATILE + raw);
        tc::tma_load_3d(sm + (size_t)s * STAGE_BYTES, &map_f, 2 * k0, row0, g.f, &full_a[s]);
      };
      auto load_raw = [&](int kt) {
        const int s = kt % STAGES, st = kb + kt;
        const int q = st / spt, k0 = (st % spt) * lp::BKC;
        const GTerm& g = tk.term[q];
        unsigned char* rawp = sm + (size_t)s * STAGE_BYTES + lp::ATILE + BTILE;
        if (g.barr) tc::tma_load_3d(rawp, &maps.b[g.barr], 2 * (tk.s0 * C + colc0), k0, g.bline, &full_a[s]);
        const int xs = 2 * ((tk.s0 + g.ds) * C + colc0);
        if (g.cpl)
          tc::tma_load_3d(rawp + lp::BASE_ROWS * RAW_ROW, &maps.s[g.arr], xs, k0 - 1, g.line, &full_a[s]);
        else
          tc::tma_load_3d(rawp + lp::BASE_ROWS * RAW_ROW, &maps.b[g.arr], xs, k0, g.line, &full_a[s]);
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
        const uint32_t a0 = smem_u32(sm + (size_t)s * STAGE_BYTES), b0 = a0 + lp::ATILE;
#pragma unroll
        for (int kk = 0; kk < 4; ++kk)  // K = 16 bf16 (32 bytes) per MMA
          lp::mma_bf16(tmem, tc::sw128_desc(a0 + kk * 32), tc::sw128_desc(b0 + kk * 32), CF::IDESC, (kt | kk) != 0);
        tc::commit(&empty[s]);
      }
      tc::commit(accfull);
      tc::griddep_launch_dependents();
    }
  } else {
    // ---------------------------------------------------------------- B builders
    const int c = threadIdx.x % BNC;   // complex column within the tile
    const int cg = threadIdx.x / BNC;  // this thread's chunks: cg, cg + CG, ... (4 nodes each)
    const bool cvalid = colc0 + c < ncols;
    const float2 vert_edge = cf.vert_f[0], vert_int = cf.vert_f[cf.n > 1 ? 1 : 0];
    const float dg = cf.diag_f;
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
      const int st = kb + kt, q = st / spt, k0 = (st % spt) * lp::BKC;
      const GTerm& g = tk.term[q];
      unsigned char* bt = sm + (size_t)s * STAGE_BYTES + lp::ATILE;
      const unsigned char* rawp = bt + BTILE;
      const float2* rb = reinterpret_cast<const float2*>(rawp);
      const float2* rs = reinterpret_cast<const float2*>(rawp + lp::BASE_ROWS * RAW_ROW);
      const float sg = g.neg ? -1.f : 1.f;
#pragma unroll
      for (int u = 0; u < CPT; ++u) {
        const int j = cg + CG * u;  // chunk: nodes 4 j .. 4 j + 3 of the stage
        uint32_t re[4], im[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int kk = 4 * j + e, k = k0 + kk;
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
          if (!(k < m && cvalid)) v = make_float2(0.f, 0.f);
          re[e] = lp::pack_bf16(v.x, -v.y);
          im[e] = lp::pack_bf16(v.y, v.x);
        }
        // every builder has read its input rows before the B area is written (the rows live
        // after it, so only this stage's own area is written: no barrier needed)
        *reinterpret_cast<uint4*>(bt + tc::sw128_off(c, j)) = make_uint4(re[0], re[1], re[2], re[3]);
        *reinterpret_cast<uint4*>(bt + tc::sw128_off(BNC + c, j)) = make_uint4(im[0], im[1], im[2], im[3]);
      }
      fence_proxy_async_smem();
      mbar_arrive(&full_b[s]);
    }

    // ---------------------------------------------------------------- epilogue
    __syncwarp();
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
      for (int qq = 0; qq < 32; qq += 2)
        *reinterpret_cast<float4*>(stile + r * SROW + 32 * h + qq) =
            ok ? make_float4(__uint_as_float(re[qq]), __uint_as_float(im[qq]), __uint_as_float(re[qq + 1]),
                             __uint_as_float(im[qq + 1]))
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
        const float2 b0 = b ? b[0] : (tk.mode == OUT_ADD ? o[0] : make_float2(0.f, 0.f));
        o[0] = make_float2(b0.x + v.x, b0.y + v.y);
        if (gc + 1 < ncols) {
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
    const unsigned nsplit = gridDim.z, qr = tc::cluster_rank();
    tc::cluster_sync();
    const int rows = (BM + (int)nsplit - 1) / (int)nsplit, r0 = (int)qr * rows;
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

// ------------------------------------------------------------------ host side
// bf16 copy of the whole complex64 factor store (round to nearest), same layout in bf16
__global__ void bf16_store_kernel(const float* __restrict__ F, __nv_bfloat16* __restrict__ B, size_t count) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
    B[i] = __float2bfloat16_rn(F[i]);
}

void set_lowp_attributes() {
  cudaFuncSetAttribute((const void*)tc_lowp_kernel<lp::Wide, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)lp::Wide::SMEM);
  cudaFuncSetAttribute((const void*)tc_lowp_kernel<lp::Wide, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)lp::Wide::SMEM);
  cudaFuncSetAttribute((const void*)tc_lowp_kernel<lp::Narrow, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)lp::Narrow::SMEM);
  cudaFuncSetAttribute((const void*)tc_lowp_kernel<lp::Narrow, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)lp::Narrow::SMEM);
}

// The bf16 factor store and its tensor map (rows of 2m bf16, m rows per block, every block;
// box 64 x 128 x 1 with the 128-byte swizzle).
int Engine::prepare_lowp() {
  if (!lowp) return HH_OK;
  auto encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(encode_fn);
  if (!encode) return (set_error("tensor-map encoder not loaded"), HH_ECUDA);
  const size_t count = (size_t)factor_blocks() * m * ldf * 2;
  if (dmalloc(&factors_bf16, count * sizeof(__nv_bfloat16))) return HH_ENOMEM;
  bf16_store_kernel<<<grid_for(count), 256, 0, stream>>>(reinterpret_cast<const float*>(factors),
                                                         reinterpret_cast<__nv_bfloat16*>(factors_bf16), count);
  count_launch();
  const cuuint64_t dims[3] = {(cuuint64_t)2 * m, (cuuint64_t)m, (cuuint64_t)factor_blocks()};
  const cuuint64_t strides[2] = {(cuuint64_t)ldf * 2 * sizeof(__nv_bfloat16),
                                 (cuuint64_t)m * ldf * 2 * sizeof(__nv_bfloat16)};
  const cuuint32_t box[3] = {64, 128, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  if (encode(&tmap_bf16, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, factors_bf16, dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return (set_error("cuTensorMapEncodeTiled failed for the bf16 factor store"), HH_ECUDA);
  const cudaError_t ce = cudaStreamSynchronize(stream);
  if (ce != cudaSuccess) return (set_cuda_error(ce, "bf16 factor store"), HH_ECUDA);
  return HH_OK;
}

// views of a sweep array with the input-row boxes of one bf16 stage, cached per (array, columns,
// tile columns, lines)
static const CUtensorMap* lowp_maps_for(Engine& E, const void* buf, int C, int bnc, int lines, bool coupled) {
  struct Ent {
    const void* ptr;
    int C, bnc, lines;
    CUtensorMap b, s;
  };
  static thread_local std::vector<Ent> cache;  // small: a handful of arrays per handle
  for (const Ent& e : cache)
    if (e.ptr == buf && e.C == C && e.bnc == bnc && e.lines == lines) return coupled ? &e.s : &e.b;
  auto encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(E.encode_fn);
  if (!encode) return nullptr;
  Ent e{buf, C, bnc, lines, {}, {}};
  const cuuint64_t dims[3] = {(cuuint64_t)2 * E.N * C, (cuuint64_t)E.m, (cuuint64_t)lines};
  const cuuint64_t strides[2] = {(cuuint64_t)2 * E.N * C * sizeof(float), (cuuint64_t)E.m * 2 * E.N * C * sizeof(float)};
  const cuuint32_t estr[3] = {1, 1, 1};
  const cuuint32_t box_b[3] = {(cuuint32_t)(2 * bnc), (cuuint32_t)lp::BASE_ROWS, 1};
  const cuuint32_t box_s[3] = {(cuuint32_t)(2 * bnc), (cuuint32_t)lp::SRC_ROWS, 1};
  void* p = const_cast<void*>(buf);
  if (encode(&e.b, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, p, dims, strides, box_b, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) !=
          CUDA_SUCCESS ||
      encode(&e.s, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, p, dims, strides, box_s, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) !=
          CUDA_SUCCESS)
    return nullptr;
  if (cache.size() >= 64) cache.erase(cache.begin());
  cache.push_back(e);
  return coupled ? &cache.back().s : &cache.back().b;
}

template <class CF>
static int run_lowp_shape(Engine& E, const std::vector<SweepPhase>& prog, const GArrays& arrs, int C) {
  LMaps maps;
  std::memset(&maps, 0, sizeof(maps));
  for (int b = SB_RIN; b < SB_COUNT; ++b) {
    if (!arrs.p[b]) continue;
    const int lines = (b == SB_T0 || b == SB_T1) ? 1 : E.R + 1;
    const CUtensorMap* mb = lowp_maps_for(E, arrs.p[b], C, CF::BNC, lines, false);
    const CUtensorMap* ms = lowp_maps_for(E, arrs.p[b], C, CF::BNC, lines, true);
    if (!mb || !ms) return (set_error("tensor maps of the sweep arrays (bf16 stages)"), HH_ECUDA);
    maps.b[b] = *mb;
    maps.s[b] = *ms;
  }
  const int gx = (E.m + tc::BM - 1) / tc::BM, spt = (E.m + lp::BKC - 1) / lp::BKC;
  for (const SweepPhase& ph : prog) {
    cudaError_t ce;
    if (ph.kind == PH_COPY) {
      ce = launch_copy_phase<float>(E, ph, arrs, C);
    } else {
      int tiles = 0, nterm = 1;
      for (const GTask& t : ph.tasks) {
        tiles += (t.ns * C + CF::BNC - 1) / CF::BNC;
        nterm = std::max(nterm, t.nterm);
      }
      const int nst = nterm * spt;
      int nsplit = std::max(1, std::min(8, (E.num_sms - 4) / (gx * tiles)));
      const int kst = (nst + nsplit - 1) / nsplit;
      nsplit = (nst + kst - 1) / kst;
      cudaLaunchConfig_t cfg{};
      cfg.gridDim = dim3(gx, tiles, nsplit);
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
      const GTask* tasks = E.pprog_tasks + ph.dev_off;
      const int ntask = (int)ph.tasks.size();
      if (nsplit > 1)
        ce = cudaLaunchKernelEx(&cfg, tc_lowp_kernel<CF, true>, E.tmap_bf16, maps, tasks, ntask, arrs, E.m, E.N, C,
                                kst, E.coef, E.err, E.opts.timeout_cycles);
      else
        ce = cudaLaunchKernelEx(&cfg, tc_lowp_kernel<CF, false>, E.tmap_bf16, maps, tasks, ntask, arrs, E.m, E.N, C,
                                kst, E.coef, E.err, E.opts.timeout_cycles);
      E.count_launch();
    }
    if (ce != cudaSuccess) return (E.set_cuda_error(ce, "bf16 sweep launch"), HH_ECUDA);
  }
  return HH_OK;
}

// One sweep with bf16 factors and products; HH_EINVAL when it cannot run that way (odd column
// count): the caller then takes the complex64 path.
int run_lowp(Engine& E, const GArrays& arrs, int C, bool single) {
  if (!E.lowp || !E.factors_bf16 || C % 2) return HH_EINVAL;
  const int d = E.depth_for(C);
  const std::vector<SweepPhase>& prog = single ? E.pprog_single_d[d] : E.pprog_double_d[d];
  if (prog.empty()) return HH_EINVAL;
  const auto it = E.tc_tuned.find(C);
  const int shape = it != E.tc_tuned.end() ? it->second.shape : 0;
  return shape == 1 ? run_lowp_shape<lp::Narrow>(E, prog, arrs, C) : run_lowp_shape<lp::Wide>(E, prog, arrs, C);
}

}  // namespace hh
