// Strip setup: block LU (Thomas) of the impedance-modified strip matrix (Section 2: a
// sweep is block forward/backward substitution of a block LU factorisation whose Schur
// complements are approximated by the impedance condition of Eq. (4)).
//
// Every strip visited before the last one has the same matrix (lines 0..R-1: facing line
// of type BOT, then R-1 lines of type INT whose far-side rows equal A's); the last strip
// has R+1 lines, its last of type TOP.  The block LU of both shares
//     S_0 = D_BOT,   S_j = D_INT - L S_{j-1}^{-1} U   (j = 1..R-1),
// and the last strip adds S_R = D_TOP - L S_{R-1}^{-1} U.  The R+1 dense inverses
// F_j = S_j^{-1} (m x m, m = n+1) are the stored factors.  L couples a line to the line
// below (vertical edge + cell diagonal), U = L^T.
//
// The inverses: complex64 blocks by Newton-Schulz (GEMMs on the tensor cores, started from the
// previous block, the Jacobi start or the scaled adjoint), pivoted Gauss-Jordan otherwise.
//
// For the sweep's interface chains (sweep.cu) setup also forms, for the strips visited
// before the last one, the first-line response of the strip inverse at its last line,
//     Y_0 = F_0,  Y_j = -F_j L Y_{j-1}   (j = 1..R-1),   Y_{R-1} = D^{-1}[R-1, 0],
// and stores G = Y_{R-1} L and K = Y_{R-1}^T U (D is complex symmetric, so
// D^{-1}[0, R-1] = Y_{R-1}^T) as blocks R+1 and R+2.
#include <cstdio>
#include <functional>
#include <vector>

#include <cmath>

#include "common.cuh"
#include "engine.h"
#include "gemm.cuh"

namespace hh {

// S = D_type - L X U  (X = previous inverse, or none for S_0); also writes column 0 of S.
template <typename R>
__global__ void schur_kernel(const typename Cx<R>::T* __restrict__ X, int ldx, int has_prev, int type,
                             Coef cf, typename Cx<R>::T* S, int ld, int m, typename Cx<R>::T* col0) {
  using T = typename Cx<R>::T;
  const size_t total = (size_t)m * m;
  const double dg = cf.diag();
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
    const int a = (int)(idx / m), b = (int)(idx % m);
    double2 d = make_double2(0.0, 0.0);
    if (a == b) d = cf.centre(a, type);
    else if (a - b == 1 || b - a == 1) d = cf.horiz(type);
    T v = mk<T>(d.x, d.y);
    if (has_prev) {
      const double2 va = cf.vert(a), vb = cf.vert(b);
      const T tva = mk<T>(va.x, va.y), tvb = mk<T>(vb.x, vb.y);
      const T tvab = cmul(tva, tvb);
      T acc = mk<T>(0, 0);
      cfma(acc, tvab, X[(size_t)a * ldx + b]);
      if (b >= 1) cfma(acc, cscale(tva, (R)dg), X[(size_t)a * ldx + b - 1]);
      if (a >= 1) cfma(acc, cscale(tvb, (R)dg), X[(size_t)(a - 1) * ldx + b]);
      if (a >= 1 && b >= 1) { T x = X[(size_t)(a - 1) * ldx + b - 1]; acc = cadd(acc, cscale(x, (R)(dg * dg))); }
      v = csub(v, acc);
    }
    S[(size_t)a * ld + b] = v;
    if (b == 0) col0[a] = v;
  }
}

// In-place Gauss-Jordan inversion with partial pivoting of one m x m complex matrix.
// Ping-pong buffers A/B (step p reads the one of parity p, writes the other); row i of the
// working matrix is owned by CTA i mod gridDim.x, 1024 threads per CTA, one column per
// thread per pass.  Column p of the source is kept contiguous in col[p & 1]; it gives the
// pivot search and every row's elimination factor.  Each thread loads its owned rows
// before the pivot search so the loads overlap it; only the pivot row is read after.
constexpr int GJ_ROWS = 8;  // owned rows per CTA held in registers per pass
template <typename R>
__global__ void __launch_bounds__(1024) gj_kernel(typename Cx<R>::T* A, typename Cx<R>::T* B,
                                                  typename Cx<R>::T* col, int* piv, int m, int ld,
                                                  unsigned* bar, int* err, long long budget) {
  using T = typename Cx<R>::T;
  __shared__ R s_val[32];
  __shared__ int s_idx[32];
  __shared__ int s_q;
  __shared__ T s_inv;
  unsigned target = 0;
  const int nw = blockDim.x >> 5, lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int G = gridDim.x;
  const int nown = (m - (int)blockIdx.x + G - 1) / G;  // rows blockIdx.x, +G, +2G, ...
  for (int p = 0; p < m; ++p) {
    const T* src = (p & 1) ? B : A;
    T* dst = (p & 1) ? A : B;
    const T* colp = col + (size_t)(p & 1) * m;
    T* coln = col + (size_t)((p + 1) & 1) * m;
    for (int r0 = 0; r0 < nown; r0 += GJ_ROWS) {
      // own rows of this pass at this thread's first column (loaded before the pivot search)
      T own[GJ_ROWS];
      {
        const int c = threadIdx.x;
#pragma unroll
        for (int r = 0; r < GJ_ROWS; ++r) {
          const int i = (int)blockIdx.x + (r0 + r) * G;
          own[r] = (c < m && r0 + r < nown) ? __ldcg(src + (size_t)i * ld + c) : mk<T>(0, 0);
        }
      }
      if (r0 == 0) {
        // pivot search over rows p..m-1 of column p
        R best = (R)-1;
        int bi = m;
        for (int i = p + threadIdx.x; i < m; i += blockDim.x) {
          const R v = cabs2(__ldcg(colp + i));
          if (v > best || (v == best && i < bi)) { best = v; bi = i; }
        }
        for (int o = 16; o; o >>= 1) {
          const R ov = __shfl_down_sync(0xffffffffu, best, o);
          const int oi = __shfl_down_sync(0xffffffffu, bi, o);
          if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
        }
        if (lane == 0) { s_val[wid] = best; s_idx[wid] = bi; }
        __syncthreads();
        if (threadIdx.x == 0) {
          for (int w = 1; w < nw; ++w)
            if (s_val[w] > best || (s_val[w] == best && s_idx[w] < bi)) { best = s_val[w]; bi = s_idx[w]; }
          s_q = bi;
          if (!(best > (R)0) || !isfinite(best)) {
            s_q = -1;
            if (blockIdx.x == 0) atomicCAS(err, 0, (int)DEV_SINGULAR);
          } else {
            const T pv = __ldcg(colp + bi);
            const R inv2 = (R)1 / cabs2(pv);
            s_inv = mk<T>(pv.x * inv2, -pv.y * inv2);
            if (blockIdx.x == 0) piv[p] = bi;
          }
        }
        __syncthreads();
      }
      const int q = s_q;
      if (q < 0) return;  // every CTA sees the same pivot column: all leave together
      const T inv = s_inv;
      for (int c = threadIdx.x; c < m; c += blockDim.x) {
        const bool first = c == (int)threadIdx.x;
        // scaled pivot row entry (old row q)
        const T prow = (c == p) ? inv : cmul(__ldcg(src + (size_t)q * ld + c), inv);
#pragma unroll
        for (int r = 0; r < GJ_ROWS; ++r) {
          if (r0 + r >= nown) continue;
          const int i = (int)blockIdx.x + (r0 + r) * G;
          T v;
          if (i == p) {
            v = prow;
          } else {
            // the working row at position i is old row i, except position q holds old row p
            const int si = (i == q) ? p : i;
            const T srow_c = (i != q && first) ? own[r] : __ldcg(src + (size_t)si * ld + c);
            const T f = __ldcg(colp + si);
            if (c == p) {
              v = cmul(f, inv);
              v.x = -v.x; v.y = -v.y;
            } else {
              v = csub(srow_c, cmul(f, prow));
            }
          }
          dst[(size_t)i * ld + c] = v;
          if (c == p + 1) coln[i] = v;
        }
      }
    }
    if (p + 1 < m) {
      if (!grid_sync(bar, target, err, budget)) return;
    }
  }
}

// Column permutation that undoes the row interchanges: F[:, c] = W[:, src[c]] where src is
// obtained by applying the interchanges (p, piv[p]) for p = m-1 down to 0.
__global__ void gj_perm_index(const int* piv, int* srcidx, int m) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    for (int c = 0; c < m; ++c) srcidx[c] = c;
    for (int p = m - 1; p >= 0; --p) {
      int q = piv[p];
      if (q < 0 || q >= m) q = p;  // an aborted inversion leaves pivots unset
      const int t = srcidx[p]; srcidx[p] = srcidx[q]; srcidx[q] = t;
    }
  }
}

template <typename R>
__global__ void gj_permute(const typename Cx<R>::T* W, int ldw, const int* srcidx, typename Cx<R>::T* F, int ldf, int m) {
  using T = typename Cx<R>::T;
  const size_t total = (size_t)m * ldf;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx / ldf), c = (int)(idx % ldf);
    F[idx] = (c < m) ? __ldcg(W + (size_t)i * ldw + srcidx[c]) : mk<T>(0, 0);
  }
}

// Z = L Y   (row a of Z couples line-node a to nodes a and a-1 of the line below)
template <typename R>
__global__ void lmul_kernel(const typename Cx<R>::T* __restrict__ Y, typename Cx<R>::T* __restrict__ Z, int m, int ld,
                            Coef cf) {
  using T = typename Cx<R>::T;
  const R dg = (R)cf.diag();
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < (size_t)m * m; idx += (size_t)gridDim.x * blockDim.x) {
    const int a = (int)(idx / m), b = (int)(idx % m);
    const double2 va = cf.vert(a);
    T v = cmul(mk<T>(va.x, va.y), Y[(size_t)a * ld + b]);
    if (a >= 1) { const T y = Y[(size_t)(a - 1) * ld + b]; v.x += dg * y.x; v.y += dg * y.y; }
    Z[(size_t)a * ld + b] = v;
  }
}

// G = Y L and K = Y^T U (L[p][p] = vert(p), L[p][p-1] = diag; U[p][p] = vert(p), U[p][p+1] = diag)
template <typename R>
__global__ void interface_kernel(const typename Cx<R>::T* __restrict__ Y, typename Cx<R>::T* __restrict__ G,
                                 typename Cx<R>::T* __restrict__ K, int m, int ld, Coef cf) {
  using T = typename Cx<R>::T;
  const R dg = (R)cf.diag();
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < (size_t)m * ld; idx += (size_t)gridDim.x * blockDim.x) {
    const int a = (int)(idx / ld), b = (int)(idx % ld);
    if (b >= m) { G[idx] = mk<T>(0, 0); K[idx] = mk<T>(0, 0); continue; }
    const double2 vb = cf.vert(b);
    const T tvb = mk<T>(vb.x, vb.y);
    T g = cmul(Y[(size_t)a * ld + b], tvb);
    if (b + 1 < m) { const T y = Y[(size_t)a * ld + b + 1]; g.x += dg * y.x; g.y += dg * y.y; }
    T k = cmul(Y[(size_t)b * ld + a], tvb);
    if (b >= 1) { const T y = Y[(size_t)(b - 1) * ld + a]; k.x += dg * y.x; k.y += dg * y.y; }
    G[idx] = g;
    K[idx] = k;
  }
}

template <typename R>
int interface_blocks(Engine& E, typename Cx<R>::T* bufA, typename Cx<R>::T* bufB) {
  using T = typename Cx<R>::T;
  const int m = E.m, ld = E.ldf, Rr = E.R;
  T* F = reinterpret_cast<T*>(E.factors);
  const size_t blk = (size_t)m * ld;
  const T* Y = F;  // Y_0 = F_0
  T* Yn[2] = {bufA, bufB};
  T* Z = nullptr;
  if (E.dmalloc((void**)&Z, blk * sizeof(T))) return HH_ENOMEM;
  for (int j = 1; j <= Rr - 1; ++j) {
    lmul_kernel<R><<<E.grid_for((size_t)m * m), 256, 0, E.stream>>>(Y, Z, m, ld, E.coef);
    E.tick_begin(Engine::K_SETUP);
    // the recursion chains R - 1 products, so it stays on the exact complex64 / complex128
    // GEMM: TF32 x 3 products here doubled the sweep's error at n = 256
    if constexpr (sizeof(R) == 4) {  // 64 x 64 tiles (33 KB of shared memory for complex64)
      dim3 grid((m + 63) / 64, (m + 63) / 64);
      dense_gemm_kernel<R, 64, 64, 4, 4><<<grid, 256, 0, E.stream>>>(F + (size_t)j * blk, ld, Z, ld, Yn[j & 1], ld, m,
                                                                     -1.0);
    } else {               // 32 x 32 tiles for complex128 (same shared memory)
      dim3 grid((m + 31) / 32, (m + 31) / 32);
      dense_gemm_kernel<R, 32, 32, 2, 2><<<grid, 256, 0, E.stream>>>(F + (size_t)j * blk, ld, Z, ld, Yn[j & 1], ld, m,
                                                                     -1.0);
    }
    E.tick_end(Engine::K_SETUP, 0.0, 8.0 * m * (double)m * m);
    E.count_launch(2);
    Y = Yn[j & 1];
  }
  interface_kernel<R><<<E.grid_for(blk), 256, 0, E.stream>>>(Y, F + (size_t)(Rr + 1) * blk, F + (size_t)(Rr + 2) * blk,
                                                             m, ld, E.coef);
  E.count_launch();
  cudaError_t ce = cudaStreamSynchronize(E.stream);
  E.dfree(Z);
  if (ce != cudaSuccess) { E.set_cuda_error(ce, "interface blocks"); return HH_ECUDA; }
  return HH_OK;
}

// Z = alpha X L (upper = 0) or alpha X U (upper = 1), with L[p][p] = vert(p), L[p][p-1] = diag,
// U[p][p] = vert(p), U[p][p+1] = diag (the couplings of a line to the line below / above);
// the padding columns of Z are zeroed.
template <typename R>
__global__ void rmul_kernel(const typename Cx<R>::T* __restrict__ X, typename Cx<R>::T* __restrict__ Z, int m, int ld,
                            Coef cf, int upper, double alpha) {
  using T = typename Cx<R>::T;
  const R dg = (R)cf.diag();
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < (size_t)m * ld; idx += (size_t)gridDim.x * blockDim.x) {
    const int a = (int)(idx / ld), b = (int)(idx % ld);
    if (b >= m) { Z[idx] = mk<T>(0, 0); continue; }
    const double2 vb = cf.vert(b);
    T v = cmul(X[(size_t)a * ld + b], mk<T>(vb.x, vb.y));
    const int nb = upper ? b - 1 : b + 1;
    if (nb >= 0 && nb < m) { const T y = X[(size_t)a * ld + nb]; v.x += dg * y.x; v.y += dg * y.y; }
    Z[idx] = mk<T>(alpha * v.x, alpha * v.y);
  }
}

// C = Eadd + alpha A B on the exact GEMM of the setup (complex64 FMA or complex128)
template <typename R>
static void exact_gemm(Engine& E, const typename Cx<R>::T* A, const typename Cx<R>::T* B, typename Cx<R>::T* C,
                       double alpha, const typename Cx<R>::T* Eadd = nullptr) {
  const int m = E.m, ld = E.ldf;
  if constexpr (sizeof(R) == 4) {
    dim3 grid((m + 63) / 64, (m + 63) / 64);
    dense_gemm_kernel<R, 64, 64, 4, 4><<<grid, 256, 0, E.stream>>>(A, ld, B, ld, C, ld, m, alpha, Eadd);
  } else {
    dim3 grid((m + 31) / 32, (m + 31) / 32);
    dense_gemm_kernel<R, 32, 32, 2, 2><<<grid, 256, 0, E.stream>>>(A, ld, B, ld, C, ld, m, alpha, Eadd);
  }
  E.count_launch();
}

// Block columns of the strip inverses and powers of the transfer blocks (the blocks of the
// sweep's interface form 1, see build_program in sweep.cu), from the stored F_j = S_j^{-1}:
//   first block column X = D^{-1} E_0 by block Thomas on the identity of line 0:
//     forward   y_0 = F_0,  y_j = -F_j L y_{j-1};
//     backward  X_top = y_top,  X_j = y_j - (F_j U) X_{j+1};
//   Y_j = X_j L for the strips visited before the last (top = R-1) and for the last (top = R);
//   last block column of the strips before the last, X = D^{-1} E_{R-1}:
//     X_{R-1} = F_{R-1},  X_j = -(F_j U) X_{j+1},  Z_j = X_j U  (j = 1..R-1, and j = 0 when
//     the twisted strip solves are stored);
//   G^(2^l) and K^(2^l) by repeated squaring.
// The products chain up to R factors, so they run on the exact GEMM (as the interface blocks).
template <typename R>
int inverse_columns_impl(Engine& E) {
  using T = typename Cx<R>::T;
  const BlockDir& bd = E.bdir;
  if (bd.iY < 0) return HH_OK;
  const int m = E.m, ld = E.ldf, Rr = E.R;
  const size_t blk = (size_t)m * ld;
  T* F = reinterpret_cast<T*>(E.factors);
  auto B = [&](int i) { return F + (size_t)i * blk; };
  T *FU = nullptr, *P[2] = {nullptr, nullptr}, *Zs = nullptr;
  if (E.dmalloc((void**)&FU, blk * sizeof(T)) || E.dmalloc((void**)&P[0], blk * sizeof(T)) ||
      E.dmalloc((void**)&P[1], blk * sizeof(T)) || E.dmalloc((void**)&Zs, blk * sizeof(T))) {
    E.dfree(FU); E.dfree(P[0]); E.dfree(P[1]); E.dfree(Zs);
    return HH_ENOMEM;
  }
  const unsigned g = E.grid_for(blk);
  auto rmul = [&](const T* X, T* Z, int upper, double alpha = 1.0) {
    rmul_kernel<R><<<g, 256, 0, E.stream>>>(X, Z, m, ld, E.coef, upper, alpha);
    E.count_launch();
  };
  int products = 0;
  E.tick_begin(Engine::K_SETUP);
  // forward: y_j in the slots of the last strip's columns
  cudaMemcpyAsync(B(bd.iYL), B(0), blk * sizeof(T), cudaMemcpyDeviceToDevice, E.stream);
  for (int j = 1; j <= Rr; ++j) {
    lmul_kernel<R><<<E.grid_for((size_t)m * m), 256, 0, E.stream>>>(B(bd.iYL + j - 1), Zs, m, ld, E.coef);
    E.count_launch();
    exact_gemm<R>(E, B(j), Zs, B(bd.iYL + j), -1.0);
    ++products;
  }
  // strips before the last: X_{R-1} = y_{R-1}
  const T* X = B(bd.iYL + Rr - 1);
  rmul(X, B(bd.iY + Rr - 1), 0);
  int pp = 0;
  for (int j = Rr - 2; j >= 0; --j) {
    rmul(B(j), FU, 1);
    T* Xn = P[pp];
    pp ^= 1;
    exact_gemm<R>(E, FU, X, Xn, -1.0, B(bd.iYL + j));
    rmul(Xn, B(bd.iY + j), 0);
    X = Xn;
    ++products;
  }
  // the last strip: X_R = y_R
  cudaMemcpyAsync(P[0], B(bd.iYL + Rr), blk * sizeof(T), cudaMemcpyDeviceToDevice, E.stream);
  X = P[0];
  pp = 1;
  rmul(X, B(bd.iYL + Rr), 0);
  for (int j = Rr - 1; j >= 0; --j) {
    rmul(B(j), FU, 1);
    T* Xn = P[pp];
    pp ^= 1;
    exact_gemm<R>(E, FU, X, Xn, -1.0, B(bd.iYL + j));
    rmul(Xn, B(bd.iYL + j), 0);
    X = Xn;
    ++products;
  }
  // last block column of the strips before the last (and Z_0 for the twisted strip solves)
  X = B(Rr - 1);
  rmul(X, B(bd.iZ + Rr - 2), 1);
  pp = 0;
  for (int j = Rr - 2; j >= (bd.iZ0 >= 0 ? 0 : 1); --j) {
    rmul(B(j), FU, 1);
    T* Xn = P[pp];
    pp ^= 1;
    exact_gemm<R>(E, FU, X, Xn, -1.0);
    rmul(Xn, j == 0 ? B(bd.iZ0) : B(bd.iZ + j - 1), 1);
    X = Xn;
    ++products;
  }
  // powers of the transfer blocks
  for (int l = 1; l < bd.LF; ++l) {
    const T* prev = l == 1 ? B(Rr + 1) : B(bd.iGp + l - 2);
    exact_gemm<R>(E, prev, prev, B(bd.iGp + l - 1), 1.0);
    ++products;
  }
  for (int l = 1; l < bd.LB; ++l) {
    const T* prev = l == 1 ? B(Rr + 2) : B(bd.iKp + l - 2);
    exact_gemm<R>(E, prev, prev, B(bd.iKp + l - 1), 1.0);
    ++products;
  }
  E.tick_end(Engine::K_SETUP, 0.0, products * 8.0 * m * (double)m * m);
  const cudaError_t ce = cudaStreamSynchronize(E.stream);
  E.dfree(FU); E.dfree(P[0]); E.dfree(P[1]); E.dfree(Zs);
  if (ce != cudaSuccess) { E.set_cuda_error(ce, "strip inverse columns"); return HH_ECUDA; }
  return E.check_device_error("strip inverse columns");
}

int Engine::inverse_columns() {
  return precision == HH_PREC_FP32 ? inverse_columns_impl<float>(*this) : inverse_columns_impl<double>(*this);
}

// Newton-Schulz step of an approximate inverse X of S (X <- X (2I - S X), quadratically
// convergent while ||I - S X||_2 < 1): with T = S X given, T is replaced by 2I - T and every
// block writes its part of ||I - T||_F^2 to part[blockIdx.x] (summed on the host in a fixed
// order, so the iteration count does not depend on the schedule).
template <typename R>
__global__ void ns_residual_kernel(typename Cx<R>::T* __restrict__ Tm, int ld, int m, double* __restrict__ part,
                                   double shift = 2.0) {
  double acc = 0;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < (size_t)m * m;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx / m), c = (int)(idx % m);
    auto& t = Tm[(size_t)i * ld + c];
    const double ex = (i == c ? 1.0 : 0.0) - (double)t.x, ey = -(double)t.y;
    acc += ex * ex + ey * ey;
    t.x = (R)((i == c ? shift : 0.0) - (double)t.x);
    t.y = -t.y;
  }
  for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  __shared__ double sh[32];
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w];
    part[blockIdx.x] = s;
  }
}

// C = A B (m x m, leading dimension ld): complex64 on the tensor cores when they are in use,
// else on the CUDA-core GEMM of the setup
template <typename R>
static void setup_gemm(Engine& E, const typename Cx<R>::T* A, const typename Cx<R>::T* B, typename Cx<R>::T* C) {
  const int m = E.m, ld = E.ldf;
  if (sizeof(R) == 4 && E.tc_dense_ok()) {
    E.tc_dense_gemm(A, B, C, false);
    return;
  }
  if constexpr (sizeof(R) == 4) {
    dim3 grid((m + 63) / 64, (m + 63) / 64);
    dense_gemm_kernel<R, 64, 64, 4, 4><<<grid, 256, 0, E.stream>>>(A, ld, B, ld, C, ld, m, 1.0);
  } else {
    dim3 grid((m + 31) / 32, (m + 31) / 32);
    dense_gemm_kernel<R, 32, 32, 2, 2><<<grid, 256, 0, E.stream>>>(A, ld, B, ld, C, ld, m, 1.0);
  }
  E.count_launch();
}

// Starting points of Newton-Schulz when the previous block is no good start.
// Jacobi: X = diag(1 / S_ii); contractive for the diagonally dominant line blocks (the first
// block of a strip is one line block, tridiagonal, ||I - S X|| about 0.5 at k = 400).
template <typename R>
__global__ void jacobi_start_kernel(const typename Cx<R>::T* __restrict__ S, int ld, int m,
                                    typename Cx<R>::T* __restrict__ X) {
  using T = typename Cx<R>::T;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < (size_t)m * m;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx / m), c = (int)(idx % m);
    T v = mk<T>(0, 0);
    if (i == c) {
      const T d = S[(size_t)i * ld + i];
      const R dd = d.x * d.x + d.y * d.y;
      v.x = d.x / dd;
      v.y = -d.y / dd;
    }
    X[(size_t)i * ld + c] = v;
  }
}
// Absolute row sums (sums[i]) and column sums (sums[m + c]) of S, for the scaled adjoint start
// (only a bound is needed: moduli in the element precision, sums in FP64).  Warp w < m sums row
// w with its lanes along the row; the threads of the remaining blocks take one column each.
template <typename R>
__global__ void abs_sums_kernel(const typename Cx<R>::T* __restrict__ S, int ld, int m, double* __restrict__ sums,
                                int row_blocks) {
  if ((int)blockIdx.x < row_blocks) {
    const int w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (w >= m) return;
    double s = 0;
    for (int c = lane; c < m; c += 32) {
      const auto v = S[(size_t)w * ld + c];
      s += (double)sqrt(v.x * v.x + v.y * v.y);
    }
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) sums[w] = s;
    return;
  }
  const int c = ((int)blockIdx.x - row_blocks) * blockDim.x + threadIdx.x;
  if (c >= m) return;
  double s = 0;
  for (int i = 0; i < m; ++i) {
    const auto v = S[(size_t)i * ld + c];
    s += (double)sqrt(v.x * v.x + v.y * v.y);
  }
  sums[m + c] = s;
}
// X = alpha S^H, alpha = 1 / (||S||_1 ||S||_inf): the eigenvalues of S X lie in (0, 1], so
// Newton-Schulz converges from it for any nonsingular S (slowly at first).
template <typename R>
__global__ void scaled_adjoint_kernel(const typename Cx<R>::T* __restrict__ S, int ld, int m, double alpha,
                                      typename Cx<R>::T* __restrict__ X) {
  using T = typename Cx<R>::T;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < (size_t)m * m;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx / m), c = (int)(idx % m);
    const T v = S[(size_t)c * ld + i];
    X[(size_t)i * ld + c] = mk<T>(alpha * v.x, -alpha * v.y);
  }
}

// F_j = S^-1 by Newton-Schulz from X_0 = F_{j-1}.  Successive Schur complements of the strip
// recursion are close (||I - S_j F_{j-1}||_2 between 0.04 and 0.14 from j = 2 on at k = 100
// and 200, cond(S_j) about 6), so a few iterations of two GEMMs replace the pivoted
// elimination.  Stops when the RMS entry of I - S X is at most 2e-7, about the complex64
// floor (or stops decreasing below 1e-4); returns false (F_j untouched beyond scratch use) when the start is not
// contractive or 16 iterations do not converge, and the caller falls back to elimination.
// With tensor cores the GEMMs are TF32 x 3 (about 2^-21 per product), which sets the floor
// the iteration stops at.
template <typename R>
static bool newton_schulz(Engine& E, const typename Cx<R>::T* S, const typename Cx<R>::T* X0, typename Cx<R>::T* Fj,
                          typename Cx<R>::T* Tb, typename Cx<R>::T* Xb, double* part_dev, double* part_host,
                          int& iters, bool from_adjoint = false) {
  using T = typename Cx<R>::T;
  const int m = E.m, ld = E.ldf;
  const int nblk = 2 * E.num_sms;
  const T* X = X0;
  T* bufs[2] = {Fj, Xb};
  double prev = 1e300;
  iters = 0;
  // from the scaled adjoint the residual need not shrink at first (its eigenvalues start near
  // 1): no contraction test, more iterations
  const int max_it = from_adjoint ? 48 : 16;
  for (int it = 0; it < max_it; ++it) {
    setup_gemm<R>(E, S, X, Tb);
    ns_residual_kernel<R><<<nblk, 256, 0, E.stream>>>(Tb, ld, m, part_dev);
    E.count_launch();
    cudaMemcpyAsync(part_host, part_dev, sizeof(double) * nblk, cudaMemcpyDeviceToHost, E.stream);
    if (cudaStreamSynchronize(E.stream) != cudaSuccess) return false;
    double s = 0;
    for (int b = 0; b < nblk; ++b) s += part_host[b];
    const double rms = std::sqrt(s / ((double)m * m));
    const bool done = rms <= 2e-7 || (rms < 1e-4 && rms > 0.5 * prev);
    if (!from_adjoint && it == 0 && std::sqrt(s) >= 0.9 * std::sqrt((double)m)) return false;  // not contractive
    if (done) {
      if (X != Fj) cudaMemcpyAsync(Fj, X, sizeof(T) * (size_t)m * ld, cudaMemcpyDeviceToDevice, E.stream);
      if constexpr (sizeof(R) == 4) {
        if (E.tc_dense_ok()) {
          // The TF32 x 3 products leave X at their floor (about 1e-6).  One refinement step
          // restores complex64 accuracy: the residual I - S X from the exact complex64 GEMM,
          // and the small correction X (I - S X) on the tensor cores added to X.
          const int m_ = E.m;
          dim3 grid((m_ + 63) / 64, (m_ + 63) / 64);
          dense_gemm_kernel<R, 64, 64, 4, 4><<<grid, 256, 0, E.stream>>>(S, ld, Fj, ld, Tb, ld, m_, 1.0);
          ns_residual_kernel<R><<<nblk, 256, 0, E.stream>>>(Tb, ld, m, part_dev, 1.0);
          E.count_launch(2);
          if (E.tc_dense_gemm(Fj, Tb, Fj, false, true) != HH_OK) return false;
        }
      }
      return true;
    }
    if (it > 2 && rms > prev && !(from_adjoint && rms > 1e-2)) return false;  // diverging
    prev = rms;
    T* Xn = bufs[it & 1];
    setup_gemm<R>(E, X, Tb, Xn);  // X (2I - S X)
    X = Xn;
    ++iters;
  }
  return false;
}

// Dense m x m line blocks for the cyclic-reduction setup: which = 0..2 the diagonal block of a
// line of type BOT / INT / TOP (tridiagonal), 3 the coupling L to the line below
// (L[a][a] = vert(a), L[a][a-1] = diag), 4 the coupling U = L^T to the line above.
template <typename R>
__global__ void line_block_kernel(typename Cx<R>::T* __restrict__ Z, int m, int ld, Coef cf, int which) {
  using T = typename Cx<R>::T;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < (size_t)m * ld; idx += (size_t)gridDim.x * blockDim.x) {
    const int a = (int)(idx / ld), b = (int)(idx % ld);
    double2 v = make_double2(0.0, 0.0);
    if (b < m) {
      if (which <= 2) {
        if (a == b) v = cf.centre(a, which);
        else if (a - b == 1 || b - a == 1) v = cf.horiz(which);
      } else {
        if (a == b) v = cf.vert(a);
        else if ((which == 3 && b == a - 1) || (which == 4 && b == a + 1)) v = make_double2(cf.diag(), 0.0);
      }
    }
    Z[idx] = mk<T>(v.x, v.y);
  }
}

// column 0 of S, contiguous (the first pivot column of the Gauss-Jordan inversion)
template <typename R>
__global__ void col0_kernel(const typename Cx<R>::T* __restrict__ S, int ld, int m, typename Cx<R>::T* __restrict__ col) {
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < m; a += gridDim.x * blockDim.x) col[a] = S[(size_t)a * ld];
}

// Inverse of one dense m x m block for the cyclic-reduction setup: complex64 by Newton-Schulz
// (from a given start, else the Jacobi start, else the scaled adjoint), then pivoted
// Gauss-Jordan as the last resort; complex128 by Gauss-Jordan.
template <typename R>
struct BlockInverter {
  using T = typename Cx<R>::T;
  Engine& E;
  T *A = nullptr, *B = nullptr, *col = nullptr, *Tb = nullptr, *Xb = nullptr, *Xs = nullptr;
  int *piv = nullptr, *srcidx = nullptr;
  double *part_dev = nullptr, *part_host = nullptr, *sums_dev = nullptr, *sums_host = nullptr;
  int inversions = 0, ns_iters = 0;
  explicit BlockInverter(Engine& e) : E(e) {}
  int alloc() {
    const size_t mat = (size_t)E.m * E.ldf * sizeof(T);
    if (E.dmalloc((void**)&A, mat) || E.dmalloc((void**)&B, mat) || E.dmalloc((void**)&col, 2 * E.m * sizeof(T)) ||
        E.dmalloc((void**)&Tb, mat) || E.dmalloc((void**)&Xb, mat) || E.dmalloc((void**)&Xs, mat) ||
        E.dmalloc((void**)&piv, E.m * sizeof(int)) || E.dmalloc((void**)&srcidx, E.m * sizeof(int)) ||
        E.dmalloc((void**)&part_dev, sizeof(double) * 2 * E.num_sms) ||
        E.dmalloc((void**)&sums_dev, sizeof(double) * 2 * E.m) ||
        cudaMallocHost((void**)&part_host, sizeof(double) * 2 * E.num_sms) != cudaSuccess ||
        cudaMallocHost((void**)&sums_host, sizeof(double) * 2 * E.m) != cudaSuccess)
      return HH_ENOMEM;
    return HH_OK;
  }
  ~BlockInverter() {
    cudaStreamSynchronize(E.stream);
    E.dfree(A); E.dfree(B); E.dfree(col); E.dfree(Tb); E.dfree(Xb); E.dfree(Xs);
    E.dfree(piv); E.dfree(srcidx); E.dfree(part_dev); E.dfree(sums_dev);
    if (part_host) cudaFreeHost(part_host);
    if (sums_host) cudaFreeHost(sums_host);
  }
  // out = S^{-1}; S is left unchanged; X0 (optional) a start close to the inverse
  int invert(const T* S, const T* X0, T* out) {
    const int m = E.m, ld = E.ldf;
    ++inversions;
    if constexpr (sizeof(R) == 4) {
      for (int start = X0 ? 0 : 1; start < 3; ++start) {
        const T* X = X0;
        if (start == 1) {
          jacobi_start_kernel<R><<<E.grid_for((size_t)m * m), 256, 0, E.stream>>>(S, ld, m, Xs);
          E.count_launch();
          X = Xs;
        } else if (start == 2) {
          const int row_blocks = (m + 7) / 8;
          abs_sums_kernel<R><<<row_blocks + (m + 255) / 256, 256, 0, E.stream>>>(S, ld, m, sums_dev, row_blocks);
          E.count_launch();
          cudaMemcpyAsync(sums_host, sums_dev, sizeof(double) * 2 * m, cudaMemcpyDeviceToHost, E.stream);
          if (cudaStreamSynchronize(E.stream) != cudaSuccess) break;
          double r1 = 0, ri = 0;
          for (int q = 0; q < m; ++q) { ri = std::max(ri, sums_host[q]); r1 = std::max(r1, sums_host[m + q]); }
          if (!(r1 > 0 && ri > 0)) break;
          scaled_adjoint_kernel<R><<<E.grid_for((size_t)m * m), 256, 0, E.stream>>>(S, ld, m, 1.0 / (r1 * ri), Xs);
          E.count_launch();
          X = Xs;
        }
        int it = 0;
        const bool ok = newton_schulz<R>(E, S, X, out, Tb, Xb, part_dev, part_host, it, start == 2);
        ns_iters += it;
        if (ok) return E.check_device_error("cyclic-reduction setup");
      }
    }
    cudaMemcpyAsync(A, S, sizeof(T) * (size_t)m * ld, cudaMemcpyDeviceToDevice, E.stream);
    col0_kernel<R><<<(m + 255) / 256, 256, 0, E.stream>>>(S, ld, m, col);
    cudaMemsetAsync(E.bar + Engine::BAR_SETUP * GRID_BAR_WORDS, 0, GRID_BAR_WORDS * sizeof(unsigned), E.stream);
    cudaMemsetAsync(piv, 0, m * sizeof(int), E.stream);
    int mm = m, ldd = ld;
    void* args[] = {(void*)&A, (void*)&B, (void*)&col, (void*)&piv, (void*)&mm, (void*)&ldd,
                    (void*)&E.bar, (void*)&E.err, (void*)&E.opts.timeout_cycles};
    const int grid = E.num_sms < m ? E.num_sms : m;
    cudaError_t ce = E.launch_coop((const void*)gj_kernel<R>, grid, 1024, 0, args);
    if (ce != cudaSuccess) { E.set_cuda_error(ce, "gj_kernel launch"); return HH_ECUDA; }
    const T* W = ((m - 1) & 1) ? A : B;
    gj_perm_index<<<1, 1, 0, E.stream>>>(piv, srcidx, m);
    gj_permute<R><<<E.grid_for((size_t)m * ld), 256, 0, E.stream>>>(W, ld, srcidx, out, ld, m);
    E.count_launch(3);
    return E.check_device_error("cyclic-reduction setup");
  }
};

// out[q] = S_q^{-1} for q = 0 .. count-1 by pivoted Gauss-Jordan in FP64, S_q formed by
// form(q, S) into one scratch block just before its inversion (it may read out[0 .. q-1]): the
// strip inverses of the five-point mode (fd.cu)
int invert_chain_fp64(Engine& E, int count, const std::function<int(int, double2*)>& form, double2* const* out) {
  BlockInverter<double> inv(E);
  if (inv.alloc()) return HH_ENOMEM;
  double2* S = nullptr;
  if (E.dmalloc((void**)&S, (size_t)E.m * E.ldf * sizeof(double2))) return HH_ENOMEM;
  cudaMemsetAsync(S, 0, (size_t)E.m * E.ldf * sizeof(double2), E.stream);
  int rc = HH_OK;
  for (int q = 0; q < count && rc == HH_OK; ++q) {
    rc = form(q, S);
    if (rc == HH_OK) rc = inv.invert(S, nullptr, out[q]);
  }
  cudaStreamSynchronize(E.stream);
  E.dfree(S);
  return rc;
}

// S = D_type - L X U - U X2 L (a null X or X2 leaves its product out), with L and U the
// couplings of a node line to the line below / above (see rmul_kernel):
//   (L X U)[a][b] = v_a v_b X[a][b] + v_a d X[a][b-1] + d v_b X[a-1][b] + d^2 X[a-1][b-1],
//   (U X L)[a][b] = v_a v_b X[a][b] + v_a d X[a][b+1] + d v_b X[a+1][b] + d^2 X[a+1][b+1],
// v = vert, d = diag: the Schur complements of the twisted strip solves.  Padding columns are
// left as they are.
template <typename R>
__global__ void schur2_kernel(const typename Cx<R>::T* __restrict__ X, const typename Cx<R>::T* __restrict__ X2,
                              int ld, int type, Coef cf, typename Cx<R>::T* __restrict__ S, int m) {
  using T = typename Cx<R>::T;
  const size_t total = (size_t)m * m;
  const R dg = (R)cf.diag();
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
    const int a = (int)(idx / m), b = (int)(idx % m);
    double2 d = make_double2(0.0, 0.0);
    if (a == b) d = cf.centre(a, type);
    else if (a - b == 1 || b - a == 1) d = cf.horiz(type);
    T v = mk<T>(d.x, d.y);
    const double2 va = cf.vert(a), vb = cf.vert(b);
    const T tva = mk<T>(va.x, va.y), tvb = mk<T>(vb.x, vb.y);
    const T tvab = cmul(tva, tvb);
    if (X) {
      T acc = mk<T>(0, 0);
      cfma(acc, tvab, X[(size_t)a * ld + b]);
      if (b >= 1) cfma(acc, cscale(tva, dg), X[(size_t)a * ld + b - 1]);
      if (a >= 1) cfma(acc, cscale(tvb, dg), X[(size_t)(a - 1) * ld + b]);
      if (a >= 1 && b >= 1) acc = cadd(acc, cscale(X[(size_t)(a - 1) * ld + b - 1], (R)(dg * dg)));
      v = csub(v, acc);
    }
    if (X2) {
      T acc = mk<T>(0, 0);
      cfma(acc, tvab, X2[(size_t)a * ld + b]);
      if (b + 1 < m) cfma(acc, cscale(tva, dg), X2[(size_t)a * ld + b + 1]);
      if (a + 1 < m) cfma(acc, cscale(tvb, dg), X2[(size_t)(a + 1) * ld + b]);
      if (a + 1 < m && b + 1 < m) acc = cadd(acc, cscale(X2[(size_t)(a + 1) * ld + b + 1], (R)(dg * dg)));
      v = csub(v, acc);
    }
    S[(size_t)a * ld + b] = v;
  }
}

// Blocks of the twisted strip solves (see append_twisted_f1 in sweep.cu): from the bottom of
// the strip matrix of lines 0..R-1 (every line below line 0 of the interior type),
//   G_{R-1} = D_int^{-1},  G_j = (D_int - U G_{j+1} L)^{-1}  (j = R-2 .. q+1),
// and the block of the meeting line q,  M = (D_int - L F_{q-1} U - U G_{q+1} L)^{-1}.
// Each inverse by Newton-Schulz from the previous block (M: from F_q), as the top-down factors.
template <typename R>
int twisted_blocks_impl(Engine& E) {
  using T = typename Cx<R>::T;
  const BlockDir& bd = E.bdir;
  if (bd.iTw < 0) return HH_OK;
  const int m = E.m, ld = E.ldf, Rr = E.R, q = bd.twq;
  const size_t blk = (size_t)m * ld;
  T* F = reinterpret_cast<T*>(E.factors);
  auto B = [&](int i) { return F + (size_t)i * blk; };
  auto G = [&](int j) { return B(bd.iTw + j - q - 1); };
  T* S = nullptr;
  if (E.dmalloc((void**)&S, blk * sizeof(T))) return HH_ENOMEM;
  cudaMemsetAsync(S, 0, blk * sizeof(T), E.stream);
  int rc = HH_OK;
  {
    BlockInverter<R> inv(E);
    rc = inv.alloc();
    const unsigned g = E.grid_for((size_t)m * m);
    E.tick_begin(Engine::K_SETUP);
    for (int j = Rr - 1; j >= q + 1 && rc == HH_OK; --j) {
      const T* prev = j == Rr - 1 ? nullptr : G(j + 1);
      schur2_kernel<R><<<g, 256, 0, E.stream>>>(nullptr, prev, ld, LINE_INT, E.coef, S, m);
      E.count_launch();
      rc = inv.invert(S, prev, G(j));
    }
    if (rc == HH_OK) {
      schur2_kernel<R><<<g, 256, 0, E.stream>>>(B(q - 1), G(q + 1), ld, LINE_INT, E.coef, S, m);
      E.count_launch();
      rc = inv.invert(S, B(q), B(bd.iTwM));
    }
    E.tick_end(Engine::K_SETUP, 0.0, 0.0);
    E.ns_blocks += inv.inversions;
    E.ns_iterations += inv.ns_iters;
  }
  const cudaError_t ce = cudaStreamSynchronize(E.stream);
  E.dfree(S);
  if (rc) return rc;
  if (ce != cudaSuccess) { E.set_cuda_error(ce, "twisted strip setup"); return HH_ECUDA; }
  return E.check_device_error("twisted strip setup");
}

int Engine::twisted_blocks() {
  return precision == HH_PREC_FP32 ? twisted_blocks_impl<float>(*this) : twisted_blocks_impl<double>(*this);
}

// Blocks of block cyclic reduction of the strip solves (see append_bcr_f1 in sweep.cu).  The
// level-0 system of a strip is block tridiagonal over its node lines: diagonal blocks D_BOT
// (line 0), D_INT, D_TOP (the last strip's line R), couplings L (to the line below) and U.
// Eliminating the odd lines of a level-(l-1) system (all of type INT) with Dinv = D_INT^{-1}
// leaves, on the even lines, the level-l system
//   D_INT' = D_INT - L Dinv U - U Dinv L,  D_BOT' = D_BOT - U Dinv L,  D_TOP' = D_TOP - L Dinv U,
//   L' = -L Dinv L,  U' = -U Dinv U;
// stored per level: Dinv, L Dinv, U Dinv (forward), Dinv L, Dinv U (back substitution).  For
// each depth d, block Thomas on the reduced system: S_0 = D_BOT^(d),
// S_i = D_INT^(d) - L^(d) F_{i-1} U^(d), S_top = D_TOP^(d) - L^(d) F_{nd-1} U^(d), F = S^{-1},
// G = F L^(d), H = F U^(d).  Products on the exact GEMM, inverses as above.
template <typename R>
int bcr_blocks_impl(Engine& E) {
  using T = typename Cx<R>::T;
  const BlockDir& bd = E.bdir;
  if (bd.dmax == 0) return HH_OK;
  const int m = E.m, ld = E.ldf;
  const size_t blk = (size_t)m * ld;
  T* F = reinterpret_cast<T*>(E.factors);
  auto B = [&](int i) { return F + (size_t)i * blk; };
  T* sc[7] = {};
  for (T*& p : sc)
    if (E.dmalloc((void**)&p, blk * sizeof(T))) {
      for (T* q : sc) E.dfree(q);
      return HH_ENOMEM;
    }
  T *Db = sc[0], *Di = sc[1], *Dt = sc[2], *Lc = sc[3], *Uc = sc[4], *T1 = sc[5], *T2 = sc[6];
  int rc = HH_OK;
  {
    BlockInverter<R> inv(E);
    rc = inv.alloc();
    const unsigned g = E.grid_for(blk);
    T* lb[5] = {Db, Di, Dt, Lc, Uc};
    for (int w = 0; w < 5 && rc == HH_OK; ++w) {
      line_block_kernel<R><<<g, 256, 0, E.stream>>>(lb[w], m, ld, E.coef, w);
      E.count_launch();
    }
    int products = 0;
    E.tick_begin(Engine::K_SETUP);
    for (int l = 1; l <= bd.dmax && rc == HH_OK; ++l) {
      const int lev = bd.iLev + 5 * (l - 1);
      T *Dinv = B(lev), *AF = B(lev + 1), *BF = B(lev + 2), *P = B(lev + 3), *Q = B(lev + 4);
      rc = inv.invert(Di, nullptr, Dinv);
      if (rc) break;
      exact_gemm<R>(E, Lc, Dinv, AF, 1.0);
      exact_gemm<R>(E, Uc, Dinv, BF, 1.0);
      exact_gemm<R>(E, Dinv, Lc, P, 1.0);
      exact_gemm<R>(E, Dinv, Uc, Q, 1.0);
      exact_gemm<R>(E, AF, Uc, Di, -1.0, Di);
      exact_gemm<R>(E, BF, Lc, Di, -1.0, Di);
      exact_gemm<R>(E, BF, Lc, Db, -1.0, Db);
      exact_gemm<R>(E, AF, Uc, Dt, -1.0, Dt);
      exact_gemm<R>(E, AF, Lc, T1, -1.0);
      exact_gemm<R>(E, BF, Uc, T2, -1.0);
      std::swap(Lc, T1);
      std::swap(Uc, T2);
      products += 10;
      if (bd.iDeep[l] < 0) continue;
      // block Thomas on the level-l system
      const int nd = E.R >> l, b = bd.iDeep[l];
      const int iF = b, iFtop = b + nd, iGtop = b + 2 * nd, iH = b + 2 * nd + 1;
      rc = inv.invert(Db, nullptr, B(iF));
      for (int i = 1; i <= nd && rc == HH_OK; ++i) {
        exact_gemm<R>(E, Lc, B(iF + i - 1), T1, 1.0);
        exact_gemm<R>(E, T1, Uc, T2, -1.0, i < nd ? Di : Dt);
        rc = inv.invert(T2, B(iF + i - 1), B(i < nd ? iF + i : iFtop));
        products += 2;
      }
      for (int i = 1; i < nd && rc == HH_OK; ++i) exact_gemm<R>(E, B(iF + i), Lc, B(b + nd + i), 1.0);
      if (rc == HH_OK) exact_gemm<R>(E, B(iFtop), Lc, B(iGtop), 1.0);
      for (int i = 0; i < nd && rc == HH_OK; ++i) exact_gemm<R>(E, B(iF + i), Uc, B(iH + i), 1.0);
      products += 2 * nd;
    }
    E.tick_end(Engine::K_SETUP, 0.0, products * 8.0 * m * (double)m * m);
  }
  const cudaError_t ce = cudaStreamSynchronize(E.stream);
  for (T* q : sc) E.dfree(q);
  if (rc) return rc;
  if (ce != cudaSuccess) { E.set_cuda_error(ce, "cyclic-reduction setup"); return HH_ECUDA; }
  return E.check_device_error("cyclic-reduction setup");
}

int Engine::bcr_blocks() {
  return precision == HH_PREC_FP32 ? bcr_blocks_impl<float>(*this) : bcr_blocks_impl<double>(*this);
}

template <typename R>
int factor_impl(Engine& E) {
  using T = typename Cx<R>::T;
  const int m = E.m, ld = E.ldf, Rr = E.R;
  T* F = reinterpret_cast<T*>(E.factors);
  T *bufA = nullptr, *bufB = nullptr, *col = nullptr;
  int *piv = nullptr, *srcidx = nullptr;
  const size_t mat = (size_t)m * ld * sizeof(T);
  if (E.dmalloc((void**)&bufA, mat) || E.dmalloc((void**)&bufB, mat) || E.dmalloc((void**)&col, 2 * m * sizeof(T)) ||
      E.dmalloc((void**)&piv, m * sizeof(int)) || E.dmalloc((void**)&srcidx, m * sizeof(int))) {
    E.dfree(bufA); E.dfree(bufB); E.dfree(col); E.dfree(piv); E.dfree(srcidx);
    return HH_ENOMEM;
  }
  int grid = E.num_sms < m ? E.num_sms : m;
  const size_t smem = 0;
  int status = HH_OK;
  // Newton-Schulz for complex64 factors (every block with the tensor cores, from the third
  // block on without; scratch: two more matrices, the residual partials and the absolute row
  // and column sums of the scaled adjoint start)
  const bool use_ns = sizeof(R) == 4;
  T *bufC = nullptr, *bufD = nullptr;
  double *part_dev = nullptr, *part_host = nullptr, *sums_dev = nullptr, *sums_host = nullptr;
  if (use_ns) {
    if (E.dmalloc((void**)&bufC, mat) || E.dmalloc((void**)&bufD, mat) ||
        E.dmalloc((void**)&part_dev, sizeof(double) * 2 * E.num_sms) ||
        E.dmalloc((void**)&sums_dev, sizeof(double) * 2 * m) ||
        cudaMallocHost((void**)&part_host, sizeof(double) * 2 * E.num_sms) != cudaSuccess ||
        cudaMallocHost((void**)&sums_host, sizeof(double) * 2 * m) != cudaSuccess) {
      E.dfree(bufA); E.dfree(bufB); E.dfree(col); E.dfree(piv); E.dfree(srcidx);
      E.dfree(bufC); E.dfree(bufD); E.dfree(part_dev); E.dfree(sums_dev);
      if (part_host) cudaFreeHost(part_host);
      if (sums_host) cudaFreeHost(sums_host);
      return HH_ENOMEM;
    }
  }
  E.ns_blocks = 0;
  E.ns_iterations = 0;
  for (int j = 0; j <= Rr && status == HH_OK; ++j) {
    const int type = (j == 0) ? LINE_BOT : (j == Rr ? LINE_TOP : LINE_INT);
    const T* X = j ? F + (size_t)(j - 1) * m * ld : nullptr;
    E.tick_begin(Engine::K_SETUP);
    schur_kernel<R><<<E.grid_for((size_t)m * m), 256, 0, E.stream>>>(X, ld, j ? 1 : 0, type, E.coef, bufA, ld, m, col);
    E.count_launch();
    if (use_ns && E.tc_dense_ok()) {
      // Newton-Schulz from the previous block, else from the Jacobi start (the first block is a
      // single line block), else from the scaled adjoint; pivoted elimination is the last resort
      int iters = 0, tried = 0;
      bool ok = false;
      for (int start = (j == 0 ? 1 : 0); start < 3 && !ok; ++start) {
        const T* X0 = X;
        if (start == 1) {
          jacobi_start_kernel<R><<<E.grid_for((size_t)m * m), 256, 0, E.stream>>>(bufA, ld, m, bufB);
          E.count_launch();
          X0 = bufB;
        } else if (start == 2) {
          const int row_blocks = (m + 7) / 8;  // 8 warps (rows) per block of 256 threads
          abs_sums_kernel<R><<<row_blocks + (m + 255) / 256, 256, 0, E.stream>>>(bufA, ld, m, sums_dev, row_blocks);
          E.count_launch();
          cudaMemcpyAsync(sums_host, sums_dev, sizeof(double) * 2 * m, cudaMemcpyDeviceToHost, E.stream);
          if (cudaStreamSynchronize(E.stream) != cudaSuccess) break;
          double r1 = 0, ri = 0;
          for (int q = 0; q < m; ++q) { ri = std::max(ri, sums_host[q]); r1 = std::max(r1, sums_host[m + q]); }
          if (!(r1 > 0 && ri > 0)) break;
          scaled_adjoint_kernel<R><<<E.grid_for((size_t)m * m), 256, 0, E.stream>>>(bufA, ld, m, 1.0 / (r1 * ri), bufB);
          E.count_launch();
          X0 = bufB;
        }
        int it_here = 0;
        ok = newton_schulz<R>(E, bufA, X0, F + (size_t)j * m * ld, bufC, bufD, part_dev, part_host, it_here, start == 2);
        iters += it_here;
        ++tried;
      }
      if (ok) {
        // 2 GEMMs per iteration, one residual GEMM per attempt, and the two of the refinement step
        E.tick_end(Engine::K_SETUP, 0.0, (2.0 * iters + tried + 2) * 8.0 * m * (double)m * m);
        ++E.ns_blocks;
        E.ns_iterations += iters;
        status = E.check_device_error("strip setup");
        continue;
      }
    } else if (use_ns && j >= 2) {
      int iters = 0;
      if (newton_schulz<R>(E, bufA, X, F + (size_t)j * m * ld, bufC, bufD, part_dev, part_host, iters)) {
        E.tick_end(Engine::K_SETUP, 0.0, (2.0 * iters + 1) * 8.0 * m * (double)m * m);
        ++E.ns_blocks;
        E.ns_iterations += iters;
        status = E.check_device_error("strip setup");
        continue;
      }
    }
    cudaMemsetAsync(E.bar + Engine::BAR_SETUP * GRID_BAR_WORDS, 0, GRID_BAR_WORDS * sizeof(unsigned), E.stream);
    cudaMemsetAsync(piv, 0, m * sizeof(int), E.stream);
    void* args[] = {(void*)&bufA, (void*)&bufB, (void*)&col, (void*)&piv, (void*)&m, (void*)&ld,
                    (void*)&E.bar, (void*)&E.err, (void*)&E.opts.timeout_cycles};
    cudaError_t ce = E.launch_coop((const void*)gj_kernel<R>, grid, 1024, smem, args);
    if (ce != cudaSuccess) { E.set_cuda_error(ce, "gj_kernel launch"); status = HH_ECUDA; break; }
    const T* W = ((m - 1) & 1) ? bufA : bufB;
    gj_perm_index<<<1, 1, 0, E.stream>>>(piv, srcidx, m);
    E.count_launch();
    gj_permute<R><<<E.grid_for((size_t)m * ld), 256, 0, E.stream>>>(W, ld, srcidx, F + (size_t)j * m * ld, ld, m);
    E.count_launch();
    E.tick_end(Engine::K_SETUP, 0.0, (double)m * m * m * 8.0);
    status = E.check_device_error("strip setup");
  }
  cudaStreamSynchronize(E.stream);
  if (status == HH_OK) status = E.check_device_error("strip setup");
  if (status == HH_OK) status = interface_blocks<R>(E, bufA, bufB);
  if (status == HH_OK) status = inverse_columns_impl<R>(E);
  if (status == HH_OK) status = bcr_blocks_impl<R>(E);
  if (status == HH_OK) status = twisted_blocks_impl<R>(E);
  E.dfree(bufA); E.dfree(bufB); E.dfree(col); E.dfree(piv); E.dfree(srcidx);
  E.dfree(bufC); E.dfree(bufD); E.dfree(part_dev); E.dfree(sums_dev);
  if (part_host) cudaFreeHost(part_host);
  if (sums_host) cudaFreeHost(sums_host);
  return status;
}

int Engine::factor() {
  return precision == HH_PREC_FP32 ? factor_impl<float>(*this) : factor_impl<double>(*this);
}

}  // namespace hh
