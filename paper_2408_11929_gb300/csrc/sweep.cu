// Batched directional double sweeps (Section 2, Eqs. (2)-(3)) as one persistent launch.
//
// Frame.  The mesh (cells cut along SW-NE diagonals) is invariant under the transpose
// (i, j) -> (j, i) and the half-turn (i, j) -> (n-i, n-j), and so is A.  The four sweeps
// are images of the bottom-to-top sweep BT under these maps (LR = transpose, TB = half
// turn, RL = both, each with its strips mapped alike, the last strip visited owning the
// extra line).  Every preconditioner application is therefore a BT sweep of a permuted
// copy of its input: the pack kernel writes each (right-hand side, direction) pair as one
// column of a line-major array X[line][node][column], one persistent kernel sweeps all
// columns together -- every factor block read once per step serves all directions and
// right-hand sides -- and the unpack kernel maps the columns back.
//
// Sweep in the BT frame, strips s = 0..N-1 of lines [sR, sR+R-1] (last: R+1 lines), with
// the block Thomas factors F_j = S_j^{-1} of the strip matrix (setup.cu):
//   forward  (strip s, j = 0..len-1): y_j = F_j (r_j - L y_{j-1})  (y_{-1}: last line of strip s-1)
//            then x_j = y_j - F_j U x_{j+1} for j = len-2..0     (v_s = x)
//   backward (strip s = N-2..0): z_{R-1} = F_{R-1} U u_{s+1}(first line),
//            z_j = F_j (-U z_{j+1}), u_j = v_j - z_j            (u_{N-1} = v_{N-1}, Section 2)
// L couples a line to the one below (vertical edge, cell diagonal), U = L^T to the one above.
#include <algorithm>
#include <cstdio>
#include <vector>

#include "common.cuh"
#include "engine.h"

namespace hh {

std::vector<SweepOp> build_schedule(int n, int N, bool double_sweep) {
  std::vector<SweepOp> ops;
  const int R = n / N;
  auto mk_op = [](int f, int out_line, int out_sub, int zsave, int base, int cpl, int src, int cline, int neg) {
    SweepOp o{};
    o.f = f; o.out_line = out_line; o.out_sub = out_sub; o.zsave = zsave; o.base_line = base;
    o.cpl = cpl; o.cpl_src = src; o.cpl_line = cline; o.cpl_neg = neg;
    return o;
  };
  for (int s = 0; s < N; ++s) {
    const int a = s * R, len = (s == N - 1) ? R + 1 : R;
    for (int j = 0; j < len; ++j) {
      const int l = a + j;
      ops.push_back(mk_op(j, l, 0, -1, l, l > 0 ? 1 : 0, 0, l - 1, 1));
    }
    for (int j = len - 2; j >= 0; --j) {
      const int l = a + j;
      ops.push_back(mk_op(j, l, 1, -1, -1, 2, 0, l + 1, 0));
    }
  }
  if (double_sweep) {
    for (int s = N - 2; s >= 0; --s) {
      const int a = s * R, b = a + R - 1;
      ops.push_back(mk_op(R - 1, b, 1, 0, -1, 2, 0, b + 1, 0));
      int slot = 0;
      for (int j = R - 2; j >= 0; --j) {
        ops.push_back(mk_op(j, a + j, 1, 1 - slot, -1, 2, 1 + slot, 0, 1));
        slot = 1 - slot;
      }
    }
  }
  return ops;
}

// BT-frame node (i, l) of a column with direction code c -> grid node (io, jo)
__device__ __forceinline__ void frame_map(int code, int i, int l, int n, int& io, int& jo) {
  switch (code) {
    case DC_BT: io = i; jo = l; break;
    case DC_TB: io = n - i; jo = n - l; break;
    case DC_LR: io = l; jo = i; break;
    default: io = n - l; jo = n - i; break;  // DC_RL
  }
}

__device__ __forceinline__ int code_of(int4 codes, int d) {
  return d == 0 ? codes.x : (d == 1 ? codes.y : (d == 2 ? codes.z : codes.w));
}

// Column-tile layout of the sweep arrays: X[line][tile][node][ct], ct = CT columns per
// tile (4 for complex64, 2 for complex128), so that one tile of one node line is a
// contiguous m * CT block that one bulk copy moves.  Columns beyond C are zero padding.
template <typename R>
__global__ void pack_kernel(const double2* const* __restrict__ srcptr, const double* __restrict__ scale, int C,
                            int t, int4 codes, int n, int ct, int ntile, typename Cx<R>::T* __restrict__ X) {
  using T = typename Cx<R>::T;
  const int m = n + 1;
  const size_t total = (size_t)m * m * ntile * ct;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
    const int cc = (int)(idx % ct);
    size_t q = idx / ct;
    const int i = (int)(q % m);
    q /= m;
    const int tile = (int)(q % ntile);
    const int l = (int)(q / ntile);
    const int c = tile * ct + cc;
    T v = mk<T>(0, 0);
    if (c < C) {
      int io, jo;
      frame_map(code_of(codes, c % t), i, l, n, io, jo);
      const double2 a = srcptr[c][(size_t)jo * m + io];
      const double s = scale[c];
      v = mk<T>(a.x * s, a.y * s);
    }
    X[idx] = v;
  }
}

template <typename R>
__global__ void unpack_kernel(const typename Cx<R>::T* __restrict__ X, int C, int t, int4 codes, int n, int ct,
                              int ntile, double2* __restrict__ dst, size_t stride) {
  const int m = n + 1;
  const size_t total = (size_t)m * m * ntile * ct;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
    const int cc = (int)(idx % ct);
    size_t q = idx / ct;
    const int i = (int)(q % m);
    q /= m;
    const int tile = (int)(q % ntile);
    const int l = (int)(q / ntile);
    const int c = tile * ct + cc;
    if (c >= C) continue;
    int io, jo;
    frame_map(code_of(codes, c % t), i, l, n, io, jo);
    dst[(size_t)c * stride + (size_t)jo * m + io] = to_d(X[idx]);
  }
}

template <typename R>
struct SweepParams {
  using T = typename Cx<R>::T;
  const T* F;        // factor blocks, m x ldf each
  const T* Rin;      // packed right-hand sides (lines x tiles x m x CT)
  T* V;              // sweep output (same layout)
  T* Zt;             // two line buffers for the backward chains
  const SweepOp* ops;
  Coef cf;
  unsigned* bar;
  int* err;
  long long budget;
  int ldf, m, ntile, nops, rp;
};

// Persistent sweep, one CTA per SM.  CTA b owns rows [b rp, (b+1) rp) of every block step.
// Per step: the CTA's rows of the factor block F_f arrive in shared memory by a bulk copy
// issued one step ahead (double buffer) so that HBM streaming overlaps the barrier; after
// the grid barrier the coupled line and the right-hand-side line arrive by bulk copy, the
// input x = Rin +- C(src) is formed in shared memory, every thread multiplies its slice of
// the node index for all of the CTA's rows and the tile's CT columns, a butterfly warp
// reduction and a cross-warp sum give the outputs, and the CTA writes its rows.
template <typename R, int CT, int RP, int NBUF>
__global__ void __launch_bounds__(256, 1) sweep_tma_kernel(SweepParams<R> p) {
  using T = typename Cx<R>::T;
  constexpr int NV = RP * CT * 2;          // real partial sums per thread
  constexpr int PER = NV / 32;             // values per lane after the butterfly
  static_assert(NV == 32 || NV == 64, "butterfly expects 32 or 64 values");
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int m = p.m, rp = p.rp, ldf = p.ldf;
  const int lineT = m * CT;
  T* Fbuf = reinterpret_cast<T*>(smem_raw);
  T* Sbuf = Fbuf + (size_t)NBUF * rp * ldf;
  T* Bbuf = Sbuf + lineT;
  T* vert_s = Bbuf + lineT;
  R* red = reinterpret_cast<R*>(vert_s + ((m + 1) & ~1));
  uint64_t* mb = reinterpret_cast<uint64_t*>(red + 8 * 64);
  __shared__ int s_ok;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int r0 = blockIdx.x * rp;
  const int nr = max(0, min(m, r0 + rp) - r0);
  const unsigned fbytes = (unsigned)(nr * ldf * sizeof(T));
  const unsigned lbytes = (unsigned)(lineT * sizeof(T));
  const size_t lstride = (size_t)p.ntile * lineT;

  for (int i = tid; i < m; i += blockDim.x) {
    const double2 v = p.cf.vert(i);
    vert_s[i] = mk<T>(v.x, v.y);
  }
  const R dg = (R)p.cf.diag();
  if (tid == 0) {
    mbar_init(&mb[0], 1);
    mbar_init(&mb[1], 1);
    mbar_init(&mb[2], 1);
    fence_proxy_async();
    if (nr > 0) {
      mbar_expect_tx(&mb[0], fbytes);
      bulk_g2s(Fbuf, p.F + (size_t)p.ops[0].f * m * ldf + (size_t)r0 * ldf, fbytes, &mb[0]);
    }
  }
  __syncthreads();
  unsigned target = 0, lphase = 0;
  for (int op = 0; op < p.nops; ++op) {
    const SweepOp o = p.ops[op];
    const int fb = (NBUF == 2) ? (op & 1) : 0;
    const unsigned fpar = (NBUF == 2) ? ((op >> 1) & 1) : (op & 1);
    if (NBUF == 2 && tid == 0 && nr > 0 && op + 1 < p.nops) {
      fence_proxy_async();
      mbar_expect_tx(&mb[(op + 1) & 1], fbytes);
      bulk_g2s(Fbuf + (size_t)((op + 1) & 1) * rp * ldf, p.F + (size_t)p.ops[op + 1].f * m * ldf + (size_t)r0 * ldf,
               fbytes, &mb[(op + 1) & 1]);
    }
    const T* src = (o.cpl_src == 0) ? p.V + (size_t)o.cpl_line * lstride : p.Zt + (size_t)(o.cpl_src - 1) * lstride;
    const T* base = o.base_line >= 0 ? p.Rin + (size_t)o.base_line * lstride : nullptr;
    T* out = p.V + (size_t)o.out_line * lstride;
    T* zs = o.zsave >= 0 ? p.Zt + (size_t)o.zsave * lstride : nullptr;
    const bool need_f = nr > 0;
    for (int tile = 0; tile < p.ntile; ++tile) {
      const unsigned nb = (o.cpl ? lbytes : 0u) + (base ? lbytes : 0u);
      if (tid == 0) {
        int ok = 1;
        if (nb) {
          fence_proxy_async();
          mbar_expect_tx(&mb[2], nb);
          if (o.cpl) bulk_g2s(Sbuf, src + (size_t)tile * lineT, lbytes, &mb[2]);
          if (base) bulk_g2s(Bbuf, base + (size_t)tile * lineT, lbytes, &mb[2]);
          ok = mbar_wait(&mb[2], lphase & 1, p.err, p.budget);
        }
        if (ok && tile == 0 && need_f) ok = mbar_wait(&mb[fb], fpar, p.err, p.budget);
        s_ok = ok;
      }
      if (nb) ++lphase;
      __syncthreads();
      if (!s_ok) return;
      // x = base +- C(src), formed in place in Bbuf
      for (int idx = tid; idx < lineT; idx += blockDim.x) {
        const int i = idx / CT;
        T v = base ? Bbuf[idx] : mk<T>(0, 0);
        if (o.cpl) {
          T cp = cmul(vert_s[i], Sbuf[idx]);
          if (o.cpl == 1 && i >= 1) { const T y = Sbuf[idx - CT]; cp.x += dg * y.x; cp.y += dg * y.y; }
          if (o.cpl == 2 && i + 1 < m) { const T y = Sbuf[idx + CT]; cp.x += dg * y.x; cp.y += dg * y.y; }
          v = o.cpl_neg ? csub(v, cp) : cadd(v, cp);
        }
        Bbuf[idx] = v;
      }
      __syncthreads();
      const T* Fr = Fbuf + (size_t)fb * rp * ldf;
      for (int g0 = 0; g0 < nr; g0 += RP) {
        const int ng = min(RP, nr - g0);
        R acc[NV];
#pragma unroll
        for (int q = 0; q < NV; ++q) acc[q] = 0;
        for (int i = tid; i < m; i += blockDim.x) {
          T xv[CT];
#pragma unroll
          for (int c = 0; c < CT; ++c) xv[c] = Bbuf[i * CT + c];
#pragma unroll
          for (int rr = 0; rr < RP; ++rr) {
            if (rr < ng) {
              const T f = Fr[(size_t)(g0 + rr) * ldf + i];
#pragma unroll
              for (int c = 0; c < CT; ++c) {
                const int q = (rr * CT + c) * 2;
                acc[q] = fma(f.x, xv[c].x, acc[q]);
                acc[q] = fma(-f.y, xv[c].y, acc[q]);
                acc[q + 1] = fma(f.x, xv[c].y, acc[q + 1]);
                acc[q + 1] = fma(f.y, xv[c].x, acc[q + 1]);
              }
            }
          }
        }
        // butterfly: after the offset-o round every lane keeps the half selected by (lane & o)
#pragma unroll
        for (int o2 = 16, half = NV / 2; o2 >= 1; o2 >>= 1, half >>= 1) {
          const bool up = (lane & o2) != 0;
#pragma unroll
          for (int q = 0; q < half; ++q) {
            const R send = up ? acc[q] : acc[q + half];
            const R keep = up ? acc[q + half] : acc[q];
            acc[q] = keep + __shfl_xor_sync(0xffffffffu, send, o2);
          }
        }
        // lane holds values [lane * PER, lane * PER + PER)
#pragma unroll
        for (int q = 0; q < PER; ++q) red[wid * 64 + lane * PER + q] = acc[q];
        __syncthreads();
        if (tid < NV / 2) {
          R re = 0, im = 0;
          for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            re += red[w * 64 + 2 * tid];
            im += red[w * 64 + 2 * tid + 1];
          }
          const int rr = tid / CT, c = tid % CT;
          if (rr < ng) {
            const size_t g = (size_t)tile * lineT + (size_t)(r0 + g0 + rr) * CT + c;
            T z;
            z.x = re;
            z.y = im;
            if (o.out_sub) out[g] = csub(__ldcg(out + g), z);
            else out[g] = z;
            if (zs) zs[g] = z;
          }
        }
        __syncthreads();
      }
    }
    if (NBUF == 1 && tid == 0 && nr > 0 && op + 1 < p.nops) {
      fence_proxy_async();
      mbar_expect_tx(&mb[0], fbytes);
      bulk_g2s(Fbuf, p.F + (size_t)p.ops[op + 1].f * m * ldf + (size_t)r0 * ldf, fbytes, &mb[0]);
    }
    if (op + 1 < p.nops) {
      if (!grid_sync(p.bar, target, p.err, p.budget)) {
        // let this CTA's outstanding factor copy land before leaving
        if (tid == 0 && nr > 0) mbar_wait(&mb[(NBUF == 2) ? ((op + 1) & 1) : 0],
                                          (NBUF == 2) ? (((op + 1) >> 1) & 1) : ((op + 1) & 1), p.err, p.budget);
        return;
      }
      if (tid == 0) fence_proxy_async();
    }
  }
}

int Engine::ensure_sweep_ws(int C) {
  const int ct = sweep_ct();
  const int ntile = (C + ct - 1) / ct;
  if ((size_t)ntile * ct <= w_cap_cols) return HH_OK;
  dfree(w_rin); dfree(w_v); dfree(w_zt);
  w_rin = w_v = w_zt = nullptr;
  w_cap_cols = 0;
  const size_t line = (size_t)m * ntile * ct * sweep_elem();
  if (dmalloc(&w_rin, line * m) || dmalloc(&w_v, line * m) || dmalloc(&w_zt, line * 2)) return HH_ENOMEM;
  w_cap_cols = (size_t)ntile * ct;
  return HH_OK;
}

// Shared memory of the sweep kernel for NBUF factor buffers.
size_t Engine::sweep_smem(int nbuf) const {
  const size_t e = sweep_elem();
  const int rp = sweep_rows_per_cta();
  return (size_t)nbuf * rp * ldf * e + 2 * (size_t)m * sweep_ct() * e + (size_t)((m + 1) & ~1) * e +
         8 * 64 * (e / 2) + 3 * sizeof(uint64_t);
}
int Engine::sweep_rows_per_cta() const { return (m + num_sms - 1) / num_sms; }
int Engine::sweep_grid() const {
  const int rp = sweep_rows_per_cta();
  return (m + rp - 1) / rp;
}

template <typename R, int CT, int NBUF>
static cudaError_t launch_sweep_t(Engine& E, const void* Rin, void* V, void* Zt, int ntile, bool single) {
  using T = typename Cx<R>::T;
  SweepParams<R> p;
  p.F = reinterpret_cast<const T*>(E.factors);
  p.Rin = reinterpret_cast<const T*>(Rin);
  p.V = reinterpret_cast<T*>(V);
  p.Zt = reinterpret_cast<T*>(Zt);
  p.ops = single ? E.d_ops_single : E.d_ops;
  p.nops = single ? E.nops_single : E.nops_double;
  p.cf = E.coef;
  p.bar = E.bar;
  p.err = E.err;
  p.budget = E.opts.timeout_cycles;
  p.ldf = E.ldf;
  p.m = E.m;
  p.ntile = ntile;
  p.rp = E.sweep_rows_per_cta();
  const size_t smem = E.sweep_smem(NBUF);
  auto fn = sweep_tma_kernel<R, CT, 8, NBUF>;
  cudaFuncSetAttribute((const void*)fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  void* args[] = {(void*)&p};
  cudaMemsetAsync(E.bar, 0, sizeof(unsigned), E.stream);
  return E.launch_coop((const void*)fn, E.sweep_grid(), 256, smem, args);
}

int Engine::run_sweep(const void* Rin, void* V, void* Zt, int C, bool single) {
  const int nops = single ? nops_single : nops_double;
  const int ct = sweep_ct();
  const int ntile = (C + ct - 1) / ct;
  const double elem = (double)sweep_elem();
  // algorithmic bytes: every block step streams one m x m factor block once for all columns,
  // the right-hand-side lines are read once and the output lines written once
  const double fbytes = (double)nops * m * m * elem + 2.0 * m * m * (double)ntile * ct * elem;
  const int nbuf = sweep_smem(2) <= 220 * 1024 ? 2 : 1;
  if (sweep_smem(nbuf) > 220 * 1024) {
    set_error("grid too large for the sweep kernel's shared-memory tiles");
    return HH_EINVAL;
  }
  tick_begin(K_SWEEP);
  cudaError_t ce;
  if (precision == HH_PREC_FP32)
    ce = nbuf == 2 ? launch_sweep_t<float, 4, 2>(*this, Rin, V, Zt, ntile, single)
                   : launch_sweep_t<float, 4, 1>(*this, Rin, V, Zt, ntile, single);
  else
    ce = nbuf == 2 ? launch_sweep_t<double, 2, 2>(*this, Rin, V, Zt, ntile, single)
                   : launch_sweep_t<double, 2, 1>(*this, Rin, V, Zt, ntile, single);
  tick_end(K_SWEEP, fbytes, (double)nops * m * m * ntile * ct * 8.0);
  last_columns = C;
  if (ce != cudaSuccess) { set_cuda_error(ce, "sweep launch"); return HH_ECUDA; }
  return HH_OK;
}

// The same launch as run_sweep without the statistics events (the no-allocation entry
// point creates no CUDA objects).
int Engine::run_sweep_untimed(const void* Rin, void* V, void* Zt, int C, bool single) {
  const int ct = sweep_ct();
  const int ntile = (C + ct - 1) / ct;
  const int nbuf = sweep_smem(2) <= 220 * 1024 ? 2 : 1;
  if (sweep_smem(nbuf) > 220 * 1024) {
    set_error("grid too large for the sweep kernel's shared-memory tiles");
    return HH_EINVAL;
  }
  cudaError_t ce;
  if (precision == HH_PREC_FP32)
    ce = nbuf == 2 ? launch_sweep_t<float, 4, 2>(*this, Rin, V, Zt, ntile, single)
                   : launch_sweep_t<float, 4, 1>(*this, Rin, V, Zt, ntile, single);
  else
    ce = nbuf == 2 ? launch_sweep_t<double, 2, 2>(*this, Rin, V, Zt, ntile, single)
                   : launch_sweep_t<double, 2, 1>(*this, Rin, V, Zt, ntile, single);
  if (ce != cudaSuccess) { set_cuda_error(ce, "sweep launch"); return HH_ECUDA; }
  return HH_OK;
}

// launch helpers used by krylov.cu / api.cu
template <typename R>
static void launch_pack_t(Engine& E, const double2* const* srcptr, const double* scale, int C, int t, int4 codes,
                          void* X) {
  const int ct = E.sweep_ct(), ntile = (C + ct - 1) / ct;
  pack_kernel<R><<<E.grid_for((size_t)E.m * E.m * ntile * ct), 256, 0, E.stream>>>(
      srcptr, scale, C, t, codes, E.n, ct, ntile, reinterpret_cast<typename Cx<R>::T*>(X));
  E.count_launch();
}
template <typename R>
static void launch_unpack_t(Engine& E, const void* X, int C, int t, int4 codes, double2* dst, size_t stride) {
  const int ct = E.sweep_ct(), ntile = (C + ct - 1) / ct;
  unpack_kernel<R><<<E.grid_for((size_t)E.m * E.m * ntile * ct), 256, 0, E.stream>>>(
      reinterpret_cast<const typename Cx<R>::T*>(X), C, t, codes, E.n, ct, ntile, dst, stride);
  E.count_launch();
}

void launch_pack(Engine& E, const double2* const* srcptr, const double* scale, int C, int t, int4 codes, void* X) {
  if (E.precision == HH_PREC_FP32) launch_pack_t<float>(E, srcptr, scale, C, t, codes, X);
  else launch_pack_t<double>(E, srcptr, scale, C, t, codes, X);
}
void launch_unpack(Engine& E, const void* X, int C, int t, int4 codes, double2* dst, size_t stride) {
  if (E.precision == HH_PREC_FP32) launch_unpack_t<float>(E, X, C, t, codes, dst, stride);
  else launch_unpack_t<double>(E, X, C, t, codes, dst, stride);
}

}  // namespace hh
