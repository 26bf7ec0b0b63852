// Complex GEMM core shared by the strip setup and the batched sweep steps.
//
//   C[:, cols] (set / -= / +=) A(m x m) * X(m x ncols)
//
// X is formed tile by tile from its sources while it is staged in shared memory:
//   * a plain matrix (setup: X = Z, row-major with leading dimension ldx), or
//   * node lines of the strip-interleaved sweep layout (sweep.cu), x = base +- C(src) where
//     C is the identity or the coupling to the line below (L) / above (U).
// A is row-major with leading dimension lda.  CTA tile BM x BN complex outputs, BK = 16,
// 256 threads, each thread TM x TN outputs accumulated in registers (no reductions).
#pragma once
#include "common.cuh"

namespace hh {

enum { XC_NONE = 0, XC_IDENT = 1, XC_LOWER = 2, XC_UPPER = 3 };
enum { OUT_SET = 0, OUT_SUB = 1, OUT_ADD = 2 };

// Layout of the sweep arrays: X[j][i][s][c] (line-in-strip j, node i, strip s, column c),
// element ((j * m + i) * N + s) * C + c.
template <typename T>
struct LineOperand {
  const T* base;   // right-hand-side array (or nullptr)
  int base_j;
  const T* src;    // coupled array (or nullptr)
  int src_j;
  int src_ds;      // strip offset of the coupled line (0, -1, +1)
  int cpl;         // XC_*
  int neg;         // x = base - C(src)
  T* out;
  int out_j, out_mode;
  T* acc;          // optional second target (nullptr)
  int acc_j, acc_mode;
  int s0, ns;      // strips
  int N, C;        // strips in the layout, columns per strip
};

template <typename T>
__device__ __forceinline__ void apply_out(T* p, T z, int mode) {
  if (mode == OUT_SET) *p = z;
  else if (mode == OUT_SUB) *p = csub(*p, z);
  else *p = cadd(*p, z);
}

template <typename R, int BM, int BN, int TM, int TN>
struct GemmTile {
  using T = typename Cx<R>::T;
  static constexpr int BK = 16;
  static_assert((BM / TM) * (BN / TN) == 256, "256 threads");
};

// cp.async of one element (8 or 16 bytes), zero-filled when !valid (src must still be a
// valid global address; callers pass the array base for invalid elements)
template <typename T>
__device__ __forceinline__ void cp_async_elem(T* dst, const T* src, bool valid) {
  static_assert(sizeof(T) == 8 || sizeof(T) == 16, "complex element");
  const unsigned d = smem_u32(dst);
  const int sz = valid ? (int)sizeof(T) : 0;
  if (sizeof(T) == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src), "r"(sz) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(d), "l"(src), "r"(sz) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Sweep step: A = factor block (m x m, row-major, lda), X formed from node lines.
// grid = (ceil(m / BM), ceil(ns * C / BN)).  Each K tile of BK node indices moves into a
// STAGES-deep ring by cp.async: the BM x BK block of A, the BK rows of the right-hand-side
// line and BK + 2 rows (one halo row each side) of the coupled line.  The tile's X is formed
// in shared memory (x = base +- C(src)), then every thread accumulates TM x TN outputs.
template <typename R, int BM, int BN, int BK, int TM, int TN, int STAGES>
__global__ void __launch_bounds__(256) line_gemm_kernel(const typename Cx<R>::T* __restrict__ A, int lda, int m,
                                                        LineOperand<typename Cx<R>::T> op, Coef cf, int kchunk,
                                                        typename Cx<R>::T* __restrict__ partial) {
  using T = typename Cx<R>::T;
  static_assert((BM / TM) * (BN / TN) == 256, "256 threads");
  constexpr int NTX = BN / TN;
  constexpr int ST_A = BM * BK, ST_B = BK * BN, ST_S = (BK + 2) * BN;
  constexpr int ST = ST_A + ST_B + ST_S;  // elements per stage
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* ring = reinterpret_cast<T*>(smem_raw);
  T* Xc = ring + (size_t)STAGES * ST;  // BK x BN formed operand
  const int tid = threadIdx.x;
  const int tx = tid % NTX, ty = tid / NTX;
  const int row0 = blockIdx.x * BM;
  const int col0 = blockIdx.y * BN;
  const int ncols = op.ns * op.C;
  const int N = op.N, C = op.C;
  const size_t istride = (size_t)N * C;  // node stride in the sweep layout
  const double2 ve = cf.vert(0), vi = cf.vert(1);
  const T vert_edge = mk<T>(ve.x, ve.y), vert_int = mk<T>(vi.x, vi.y);
  const R dg = (R)cf.diag();
  const bool has_base = op.base != nullptr, has_src = op.cpl != XC_NONE;
  // column gc of this step = strip s0 + gc / C, column gc % C: address offset within a node row
  const T* base_row0 = has_base ? op.base + ((size_t)op.base_j * m * N + op.s0) * C : nullptr;
  const T* src_row0 = has_src ? op.src + ((size_t)op.src_j * m * N + op.s0 + op.src_ds) * C : nullptr;
  // split K: this CTA covers node indices [kbeg, kend)
  const int kbeg = blockIdx.z * kchunk;
  const int kend = min(m, kbeg + kchunk);

  auto issue = [&](int stage, int k0) {
    T* As = ring + (size_t)stage * ST;
    T* Bb = As + ST_A;
    T* Bs = Bb + ST_B;
    for (int e = tid; e < BM * BK; e += 256) {
      const int r = e / BK, kk = e % BK;
      const int gr = row0 + r, gk = k0 + kk;
      const bool v = gr < m && gk < kend;
      cp_async_elem(As + r * BK + kk, A + (size_t)(v ? gr : 0) * lda + (v ? gk : 0), v);
    }
    if (has_base)
      for (int e = tid; e < BK * BN; e += 256) {
        const int kk = e / BN, cc = e % BN;
        const int gk = k0 + kk, gc = col0 + cc;
        const bool v = gk < m && gc < ncols;
        cp_async_elem(Bb + e, base_row0 + (v ? (size_t)gk * istride + gc : 0), v);
      }
    if (has_src)
      for (int e = tid; e < (BK + 2) * BN; e += 256) {
        const int rr = e / BN, cc = e % BN;
        const int gk = k0 + rr - 1, gc = col0 + cc;
        const bool v = gk >= 0 && gk < m && gc < ncols;
        cp_async_elem(Bs + e, src_row0 + (v ? (size_t)gk * istride + gc : 0), v);
      }
  };

  R acc[TM][TN][2];
#pragma unroll
  for (int a = 0; a < TM; ++a)
#pragma unroll
    for (int b = 0; b < TN; ++b) acc[a][b][0] = acc[a][b][1] = 0;

  const int nk = kend > kbeg ? (kend - kbeg + BK - 1) / BK : 0;
#pragma unroll
  for (int s = 0; s < STAGES - 1; ++s) {
    if (s < nk) issue(s, kbeg + s * BK);
    cp_async_commit();
  }
  for (int kt = 0; kt < nk; ++kt) {
    cp_async_wait<STAGES - 2>();
    __syncthreads();
    const int stage = kt % STAGES;
    const T* As = ring + (size_t)stage * ST;
    const T* Bb = As + ST_A;
    const T* Bs = Bb + ST_B;
    const int k0 = kbeg + kt * BK;
    for (int e = tid; e < BK * BN; e += 256) {
      const int kk = e / BN, cc = e % BN;
      const int gk = k0 + kk;
      T v = has_base ? Bb[e] : mk<T>(0, 0);
      if (has_src) {
        T cp = Bs[(kk + 1) * BN + cc];
        if (op.cpl != XC_IDENT) {
          cp = cmul((gk == 0 || gk == m - 1) ? vert_edge : vert_int, cp);
          const T y = Bs[(op.cpl == XC_LOWER ? kk : kk + 2) * BN + cc];  // zero outside the grid
          cp.x += dg * y.x;
          cp.y += dg * y.y;
        }
        v = op.neg ? csub(v, cp) : cadd(v, cp);
      }
      Xc[e] = v;
    }
    __syncthreads();
    {
      const int nt = kt + STAGES - 1;
      if (nt < nk) issue(nt % STAGES, kbeg + nt * BK);
      cp_async_commit();
    }
#pragma unroll 8
    for (int kk = 0; kk < BK; ++kk) {
      T a[TM], x[TN];
#pragma unroll
      for (int q = 0; q < TM; ++q) a[q] = As[(ty * TM + q) * BK + kk];
#pragma unroll
      for (int q = 0; q < TN; ++q) x[q] = Xc[kk * BN + tx * TN + q];
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
  }
  cp_async_wait<0>();
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
      if (partial) {  // split K: the reduce kernel sums the slices and applies the outputs
        partial[((size_t)blockIdx.z * m + gr) * ncols + gc] = z;
        continue;
      }
      const int s = op.s0 + gc / C, c = gc % C;
      T* o = op.out + ((size_t)(op.out_j * m + gr) * N + s) * C + c;
      apply_out(o, z, op.out_mode);
      if (op.acc) {
        T* a2 = op.acc + ((size_t)(op.acc_j * m + gr) * N + s) * C + c;
        apply_out(a2, op.out_mode == OUT_SET ? z : *o, op.acc_mode);
      }
    }
  }
}

// Sum of the split-K slices in a fixed order, then the step's output modes.
template <typename R>
__global__ void split_reduce_kernel(const typename Cx<R>::T* __restrict__ partial, int nsplit, int m,
                                    LineOperand<typename Cx<R>::T> op) {
  using T = typename Cx<R>::T;
  // Launched with programmatic dependent launch after a tensor-core step: the next step may
  // start its prologue at once, and this grid waits until the step that wrote the slices has
  // completed (both are no-ops for a plain launch).
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  asm volatile("griddepcontrol.wait;" ::: "memory");
  const int ncols = op.ns * op.C;
  const size_t total = (size_t)m * ncols;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
    T z = partial[idx];
    for (int k = 1; k < nsplit; ++k) z = cadd(z, partial[(size_t)k * total + idx]);
    const int gr = (int)(idx / ncols), gc = (int)(idx % ncols);
    const int s = op.s0 + gc / op.C, c = gc % op.C;
    T* o = op.out + ((size_t)(op.out_j * m + gr) * op.N + s) * op.C + c;
    apply_out(o, z, op.out_mode);
    if (op.acc) {
      T* a2 = op.acc + ((size_t)(op.acc_j * m + gr) * op.N + s) * op.C + c;
      apply_out(a2, op.out_mode == OUT_SET ? z : *o, op.acc_mode);
    }
  }
}

template <typename R, int BM, int BN, int BK, int STAGES>
constexpr size_t line_gemm_smem() {
  return ((size_t)STAGES * (BM * BK + BK * BN + (BK + 2) * BN) + BK * BN) * sizeof(typename Cx<R>::T);
}

// Setup GEMM: C = E + alpha * A * B (all m x m, row-major, leading dimensions lda / ldb / ldc;
// E optional, with leading dimension ldc, and it may be C itself).
// The next K tile is copied into the other shared-memory buffer by cp.async while the current
// one is multiplied (two buffers, one copy group in flight).
template <typename R, int BM, int BN, int TM, int TN>
__global__ void __launch_bounds__(256) dense_gemm_kernel(const typename Cx<R>::T* __restrict__ A, int lda,
                                                         const typename Cx<R>::T* __restrict__ B, int ldb,
                                                         typename Cx<R>::T* Cm, int ldc, int m,
                                                         double alpha, const typename Cx<R>::T* E = nullptr) {
  using T = typename Cx<R>::T;
  constexpr int BK = 16;
  constexpr int NTX = BN / TN;
  __shared__ __align__(16) T As[2][BK][BM + 1];
  __shared__ __align__(16) T Bs[2][BK][BN];
  const int tid = threadIdx.x;
  const int tx = tid % NTX, ty = tid / NTX;
  const int row0 = blockIdx.x * BM;
  const int col0 = blockIdx.y * BN;
  auto load_tile = [&](int buf, int k0) {
    for (int e = tid; e < BK * BM; e += 256) {
      const int r = e / BK, kk = e % BK;  // consecutive threads walk along a row of A
      const int gr = row0 + r, gk = k0 + kk;
      const bool ok = gr < m && gk < m;
      cp_async_elem(&As[buf][kk][r], ok ? A + (size_t)gr * lda + gk : A, ok);
    }
    for (int e = tid; e < BK * BN; e += 256) {
      const int kk = e / BN, cc = e % BN;
      const int gk = k0 + kk, gc = col0 + cc;
      const bool ok = gk < m && gc < m;
      cp_async_elem(&Bs[buf][kk][cc], ok ? B + (size_t)gk * ldb + gc : B, ok);
    }
    cp_async_commit();
  };
  R acc[TM][TN][2];
#pragma unroll
  for (int a = 0; a < TM; ++a)
#pragma unroll
    for (int b = 0; b < TN; ++b) acc[a][b][0] = acc[a][b][1] = 0;
  const int nk = (m + BK - 1) / BK;
  load_tile(0, 0);
  for (int kt = 0; kt < nk; ++kt) {
    const int cur = kt & 1;
    // tile kt has landed, and every thread is done with tile kt - 1, whose buffer is refilled
    cp_async_wait<0>();
    __syncthreads();
    if (kt + 1 < nk) load_tile(cur ^ 1, (kt + 1) * BK);
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T a[TM], x[TN];
#pragma unroll
      for (int q = 0; q < TM; ++q) a[q] = As[cur][kk][ty * TM + q];
#pragma unroll
      for (int q = 0; q < TN; ++q) x[q] = Bs[cur][kk][tx * TN + q];
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
  }
#pragma unroll
  for (int p = 0; p < TM; ++p) {
    const int gr = row0 + ty * TM + p;
    if (gr >= m) continue;
#pragma unroll
    for (int q = 0; q < TN; ++q) {
      const int gc = col0 + tx * TN + q;
      if (gc >= m) continue;
      T z = mk<T>(alpha * acc[p][q][0], alpha * acc[p][q][1]);
      if (E) z = cadd(E[(size_t)gr * ldc + gc], z);
      Cm[(size_t)gr * ldc + gc] = z;
    }
  }
}

}  // namespace hh
