// Block Gram-Schmidt against the basis on the tensor cores, to FP64 accuracy (Section 3's
// inner products H = V^H W and update W -= V H of every CGS pass).
//
// GB300's FP64 pipe runs at about 1/64 of its FP32 rate, and the FP64 kernels of these two
// products (krylov.cu) are bound by it.  Here both are exact integer GEMMs on the bf16 tensor
// cores, in the manner of the Ozaki splitting:
//
//   * a real vector x with max |x| < 2^e is written as x = 2^e sum_{i<8} s_i 2^{-7(i+1)} + err,
//     |err| < 2^{e-56}, with integer digits |s_i| <= 127 (sign-magnitude, from the FP64 bits:
//     no floating-point arithmetic), each held exactly in bf16 (8 significant bits);
//   * a product of two digits is below 2^14 in magnitude, so 1024 of them sum exactly in the
//     FP32 accumulator of tcgen05.mma.kind::f16 (below 2^24); every accumulator is read out
//     after at most 1024 products and its digit-pair weights applied in FP64.
// The result carries the rounding of the FP64 combination only (a few units of 2^-53 of
// sum |v||w|), plus the digit truncation (2^-56 of max |v| max |w| per term).
//
// Complex data as real GEMMs, with c = 0 / 1 the real / imaginary plane:
//   inner products  Re <v, w> = sum_c sum_g v_c w_c,  Im <v, w> = sum_g v_0 w_1 - v_1 w_0,
//     so the new column w_b gives two rows of the B operand: (w_0, w_1) and (w_1, -w_0);
//   update          (V H)_c = sum_a sum_c' v_{a,c'} G[a, c', (b, c)] with G[a,0,(b,0)] = Re h,
//     G[a,1,(b,0)] = -Im h, G[a,0,(b,1)] = Im h, G[a,1,(b,1)] = Re h.
//
// Data (per basis vector, written once when the vector is accepted, 64 Dp bytes; Dp = node
// count padded to a multiple of 768):
//   DI  the "dot image": for plane c and node chunk q (64 nodes), 1 KB = 8 rows (digit i) of 64
//       bf16, 128-byte swizzled (a K-major SW128 atom of the MMA's A operand);
//   NI  the "node image": for every 128-node tile, 4 KB = 128 rows (node) of 16 bf16 (plane c,
//       digit i), K-major without swizzle: 8x8 core matrices, cores along K 128 B apart, 8-row
//       groups 256 B apart.
// Per pass: the new columns' B operand of the inner products (rows (b, part, digit j), 64 nodes
// per 128-byte row, SW128), formed in shared memory by the inner-product kernel from W itself,
// and the coefficient image CB of every basis vector (B
// operand of the update: rows (b, part, weight group w), K = (plane, digit i), value digit
// w - i of G 2^{e_a} when 0 <= w - i < 8; pairs of weight group w >= 10, 2^-70 of the leading
// pair and below, are dropped).
//
// Kernels: gst_dot_kernel (one CTA per SM, a contiguous node range each; stages of 128 nodes,
// one 2 KB copy per basis vector, the new columns' digits sliced from W by four warps of the
// CTA; rows (vector, digit) of up to 8 tiles of 16 vectors in
// tensor memory, read out every 1024 products and summed exactly in int64), gst_upd_kernel
// (persistent over tiles of 384 nodes; per basis vector one 12 KB node-image copy and three
// MMAs of M = 128 nodes, N = rows of CB, K = 16; accumulators read out after every 64
// vectors, double-buffered in tensor memory).  Operand tiles arrive by cp.async.bulk (the
// images are stored in the MMA's shared-memory layout).  Every wait is bounded (E.err,
// opts.timeout_cycles).  The per-flush arithmetic uses integer instructions only: GB300's
// FP64 pipe, which also takes 64-bit conversions, is the resource this file avoids.
#include <algorithm>
#include <cstdio>
#include <vector>

#include <cuda_bf16.h>

#include "common.cuh"
#include "engine.h"
#include "kstate.h"
#include "tc_gemm.cuh"

namespace hh {
namespace gst {

constexpr int SL = 8;          // digits per value
// inner products: warp 0 producer, warp 1 MMA + tensor memory, warps 2-5 epilogue, warps 6-9
// slicer (the new columns' B operand, formed from W in shared memory)
constexpr int THREADS = 320;
constexpr int EPI_THREADS = 128;
constexpr int SLICE_THREADS = 128;  // one node of the stage's 128 each
// inner products
constexpr int DOT_SC = 2;      // 64-node chunks per stage (one 2 KB copy per basis vector)
constexpr int DOT_NA = 4;      // A ring: 32 KB tiles (16 vectors x 8 digits x 128 nodes)
constexpr int DOT_NB = 3;      // B ring: the new columns' digits of a stage (two 64-node blocks)
constexpr int DOT_FL = 16 / DOT_SC;  // stages per exact accumulation period (1024 products)
constexpr int DOT_MAXT = 8;    // tiles per tensor-memory round (8 x 16 t columns <= 512)
constexpr int ATILE = 16 * DOT_SC * 1024;
// update
constexpr int UPD_PARTS = 3;   // 128-node parts per tile (one MMA each)
constexpr int UPD_NS = 12;     // ring stages: the parts' node images + one coefficient image
constexpr int UPD_SEG = 64;    // basis vectors per exact accumulation period (64 x 16 products)
constexpr int UPD_NODES = 128 * UPD_PARTS;   // nodes per tile
constexpr int UPD_THREADS = 64 + 128 * UPD_PARTS;  // producer, MMA, four epilogue warps per part

__host__ __device__ constexpr int nu_rows(int t) { return (20 * t + 15) / 16 * 16; }
__host__ __device__ constexpr int dot_bbytes(int t) { return 16 * t * 128; }
__host__ __device__ constexpr int upd_stage_bytes(int t) {
  return (4096 * UPD_PARTS + nu_rows(t) * 32 + 1023) / 1024 * 1024;
}
constexpr int DOT_CONV = 128; // flushes between conversions of the int64 sums to FP64
constexpr int PTR_CACHE = 1024; // basis-vector image pointers kept in shared memory
constexpr size_t dot_smem(int t) {
  return 1024 + (size_t)DOT_NA * ATILE + (size_t)DOT_NB * DOT_SC * dot_bbytes(t) + (size_t)DOT_MAXT * 16 * 2 * t * 8 * 3 +
         (2 * DOT_NA + 2 * DOT_NB + 2 * DOT_MAXT + 1) * 8 + PTR_CACHE * 8;
}
constexpr size_t upd_smem(int t) {
  return 1024 + (size_t)UPD_NS * upd_stage_bytes(t) + (2 * UPD_NS + 5) * 8 + PTR_CACHE * 8;
}

// An integer-valued FP32 accumulator (|f| < 2^24) as int, from its bits (ALU instructions only:
// a conversion instruction whose result feeds 64-bit arithmetic can be issued to the FP64 pipe)
__device__ __forceinline__ int f2i_exact(float f) {
  const int b = __float_as_int(f);
  const int sh = 150 - ((b >> 23) & 0xFF);  // |f| = m 2^-sh, m the 24-bit significand
  const int v = sh < 24 ? (((b & 0x7FFFFF) | 0x800000) >> sh) : 0;
  return b < 0 ? -v : v;
}

// v 2^e as FP64 (|v| < 2^62), rounded to nearest (ties away from zero), with integer
// instructions only (GB300's FP64 pipe is the scarce one; int64 ->
// FP64 conversion and ldexp run on it)
__device__ __forceinline__ double i64_scaled(long long v, int e) {
  if (v == 0) return 0.0;
  const unsigned long long sgn = v < 0 ? (1ull << 63) : 0ull;
  unsigned long long a = v < 0 ? (unsigned long long)(-v) : (unsigned long long)v;
  int msb = 63 - __clzll((long long)a);
  if (msb > 52) {
    a += 1ull << (msb - 53);  // half a unit of the last kept bit; may carry into a new top bit
    msb = 63 - __clzll((long long)a);
  }
  const unsigned long long m = msb >= 52 ? a >> (msb - 52) : a << (52 - msb);
  const int ex = msb + e + 1023;
  // below the normal range: zero (under 2^-1022); above it: infinity.  No FP64 fallback: a
  // branch to one is predicated into the straight-line code and occupies the FP64 pipe.
  if (ex <= 0) return __longlong_as_double((long long)sgn);
  if (ex >= 2047) return __longlong_as_double((long long)(sgn | (0x7FFull << 52)));
  return __longlong_as_double((long long)(sgn | ((unsigned long long)ex << 52) | (m & ((1ull << 52) - 1))));
}

// exponent e of frexp(x) for the bits of |x| (x = f 2^e, 1/2 <= f < 1): |x| < 2^e; 0 for x = 0;
// INT_MAX when x is not finite
__host__ __device__ __forceinline__ int frexp_exp_bits(unsigned long long b) {
  const int ex = (int)((b >> 52) & 0x7FF);
  if (ex == 0x7FF) return 0x7FFFFFFF;
  if (ex == 0) return b ? -1021 : 0;  // subnormal: below 2^-1021
  return ex - 1022;
}

// the eight signed 7-bit digits of x 2^-e (|x| < 2^e), truncated: |x 2^-e - sum d_i 2^{-7(i+1)}|
// < 2^-56.  Subnormal x count as zero.
__device__ __forceinline__ void digits8(double x, int e, int (&d)[SL]) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
  const int ex = (int)((bits >> 52) & 0x7FF);
  unsigned long long F = 0;
  if (ex != 0) {
    const unsigned long long mant = (bits & ((1ull << 52) - 1)) | (1ull << 52);
    // |x| = mant 2^(ex - 1075);  F = floor(|x| 2^(56 - e)) < 2^56
    const int sh = ex - 1075 + 56 - e;
    F = sh >= 0 ? (mant << sh) : (sh > -64 ? (mant >> -sh) : 0ull);
  }
  const bool neg = (bits >> 63) != 0;
#pragma unroll
  for (int i = 0; i < SL; ++i) {
    const int v = (int)((F >> (49 - 7 * i)) & 127ull);
    d[i] = neg ? -v : v;
  }
}

__device__ __forceinline__ uint32_t bf16x2(int lo, int hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn((float)lo, (float)hi);  // exact: |digit| <= 127
  return *reinterpret_cast<const uint32_t*>(&v);
}

// byte offset of 16-byte chunk (row r, K core kc) in a no-swizzle K-major image with two K cores
__host__ __device__ __forceinline__ uint32_t ns_off(int r, int kc) {
  return (uint32_t)(((r >> 3) * 2 + kc) * 128 + (r & 7) * 16);
}

__device__ __forceinline__ unsigned long long abs_bits(double x) {
  return (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull;
}

}  // namespace gst

// ------------------------------------------------------------------ slicing kernels
namespace {

__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    const unsigned long long u = __shfl_xor_sync(0xffffffffu, v, o);
    v = u > v ? u : v;
  }
  return v;
}

// max |entry| (as the bits of the FP64 magnitude, ordered like the values) of the basis vectors
// still to be sliced.  Grid (GX, slots, t); mode 1: only the slots being admitted.
__global__ void gst_vscan_kernel(KState S, int mode) {
  const int r = blockIdx.y, q = blockIdx.z;
  if (mode ? !S.adm[r] : false) return;
  const int a = S.vnew0[r] + q;
  if (a >= S.vnew1[r]) return;
  const double2* v = S.Vptr[(size_t)r * S.maxV + a];
  unsigned long long m = 0;
  for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < (size_t)S.D; g += (size_t)gridDim.x * blockDim.x) {
    const double2 x = v[g];
    const unsigned long long b0 = gst::abs_bits(x.x), b1 = gst::abs_bits(x.y);
    m = b0 > m ? b0 : m;
    m = b1 > m ? b1 : m;
  }
  m = warp_max_u64(m);
  if ((threadIdx.x & 31) == 0 && m) atomicMax(&S.vmaxb[(size_t)r * S.t + q], m);
}

// The dot and node images of the basis vectors still to be sliced (one thread per node,
// nodes D .. Dp-1 written as zeros; a CTA takes 256 nodes, its four 1 KB dot-image chunks of
// each plane placed in shared memory and written out with 16-byte stores).  Grid (blocks over
// Dp / 256, slots, t).
__global__ void __launch_bounds__(256) gst_vslice_kernel(KState S, int mode) {
  const int r = blockIdx.y, q = blockIdx.z;
  if (mode ? !S.adm[r] : false) return;
  const int a = S.vnew0[r] + q;
  if (a >= S.vnew1[r]) return;
  __shared__ __align__(16) unsigned char dsm[2 * 4 * 1024];
  const int e = gst::frexp_exp_bits(S.vmaxb[(size_t)r * S.t + q]);
  if (blockIdx.x == 0 && threadIdx.x == 0) S.vexp[(size_t)r * S.maxV + a] = e;
  const double2* v = S.Vptr[(size_t)r * S.maxV + a];
  unsigned char* DI = S.VSptr[(size_t)r * S.maxV + a];
  unsigned char* NI = DI + (size_t)32 * S.Dp;
  const size_t chunks = (size_t)S.Dp / 64;
  for (size_t g0 = (size_t)blockIdx.x * 256; g0 < (size_t)S.Dp; g0 += (size_t)gridDim.x * 256) {
    const size_t g = g0 + threadIdx.x;
    int d[2][gst::SL];
    const double2 x = (g < (size_t)S.D && e != 0x7FFFFFFF) ? v[g] : make_double2(0, 0);
    gst::digits8(x.x, e, d[0]);
    gst::digits8(x.y, e, d[1]);
    const int kk = threadIdx.x & 63, qq = threadIdx.x >> 6;
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      unsigned char* blk = dsm + (c * 4 + qq) * 1024;
#pragma unroll
      for (int i = 0; i < gst::SL; ++i)
        *reinterpret_cast<__nv_bfloat16*>(blk + i * 128 + ((((kk >> 3) ^ i)) << 4) + (kk & 7) * 2) =
            __float2bfloat16_rn((float)d[c][i]);
      *reinterpret_cast<uint4*>(NI + (g >> 7) * 4096 + gst::ns_off((int)(g & 127), c)) =
          make_uint4(gst::bf16x2(d[c][0], d[c][1]), gst::bf16x2(d[c][2], d[c][3]), gst::bf16x2(d[c][4], d[c][5]),
                     gst::bf16x2(d[c][6], d[c][7]));
    }
    __syncthreads();
    const size_t q0 = g0 / 64;
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      uint4* dst = reinterpret_cast<uint4*>(DI + ((size_t)c * chunks + q0) * 1024);
      const uint4* src = reinterpret_cast<const uint4*>(dsm + c * 4 * 1024);
      dst[threadIdx.x] = src[threadIdx.x];  // 4 KB = 256 x 16 bytes
    }
    __syncthreads();
  }
}

// max |entry| of every new column, and (first pass) this CTA's part of |A z_j|^2, the deflation
// reference of the block QR (same layout as gs_wprep_kernel's).  Grid (GX, slots).
template <int TT>
__global__ void __launch_bounds__(256) gst_wscan_kernel(KState S, const double2* __restrict__ W, int first) {
  const int r = blockIdx.y;
  if (S.done[r]) return;
  const size_t D = S.D;
  const double2* Wr = W + (size_t)r * TT * D;
  unsigned long long m[TT];
  double n2[TT];
#pragma unroll
  for (int b = 0; b < TT; ++b) { m[b] = 0; n2[b] = 0; }
  for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < D; g += (size_t)gridDim.x * blockDim.x) {
#pragma unroll
    for (int b = 0; b < TT; ++b) {
      const double2 w = Wr[b * D + g];
      const unsigned long long b0 = gst::abs_bits(w.x), b1 = gst::abs_bits(w.y);
      m[b] = b0 > m[b] ? b0 : m[b];
      m[b] = b1 > m[b] ? b1 : m[b];
      n2[b] += w.x * w.x + w.y * w.y;
    }
  }
  __shared__ double sh[8][TT];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int b = 0; b < TT; ++b) {
    m[b] = warp_max_u64(m[b]);
    if (lane == 0 && m[b]) atomicMax(&S.wmaxb[(size_t)r * TT + b], m[b]);
    double s = n2[b];
#pragma unroll
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) sh[wid][b] = s;
  }
  if (!first) return;
  __syncthreads();
  if (threadIdx.x < TT) {
    double s = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w][threadIdx.x];
    S.azpart[((size_t)r * TT + threadIdx.x) * gridDim.x + blockIdx.x] = s;
  }
}

// Coefficient images CB of this pass's H (one CTA per slot): per new column b the exponent E_b
// with max_a |h_ab 2^{e_a}| < 2^{E_b} (a scale per output column keeps each column's update
// relative to its own coefficients), then for every basis vector a the rows
// n = (2 b + part) 10 + w of its image (K = plane c x digit i: digit w - i of
// G[a, c, (b, part)] 2^{e_a - E_b}).
template <int TT>
__global__ void __launch_bounds__(256) gst_cslice_kernel(KState S) {
  const int r = blockIdx.x;
  if (S.done[r]) return;
  const int p = S.nV[r], NU = S.NU;
  const double2* H = S.Hthis + (size_t)r * S.maxV * TT;
  const int* vexp = S.vexp + (size_t)r * S.maxV;
  __shared__ int shm[8][TT];
  __shared__ int Es[TT];
  // per column b: max over a of |h_ab| 2^{e_a}, as an exponent (the exponent of |h| plus e_a)
  int emax[TT];
  bool bad = false;
#pragma unroll
  for (int b = 0; b < TT; ++b) emax[b] = -0x7FFFFFFF;
  for (int a = threadIdx.x; a < p; a += blockDim.x) {
    const int ea = vexp[a];
#pragma unroll
    for (int b = 0; b < TT; ++b) {
      const double2 h = H[(size_t)a * TT + b];
      const unsigned long long bm = max(gst::abs_bits(h.x), gst::abs_bits(h.y));
      const int eh = gst::frexp_exp_bits(bm);
      if (eh == 0x7FFFFFFF) bad = true;
      else if (bm) emax[b] = max(emax[b], eh + ea);
    }
  }
#pragma unroll
  for (int b = 0; b < TT; ++b)
    for (int o = 16; o; o >>= 1) emax[b] = max(emax[b], __shfl_xor_sync(0xffffffffu, emax[b], o));
  const int anybad = __syncthreads_or(bad ? 1 : 0);
  if ((threadIdx.x & 31) == 0)
#pragma unroll
    for (int b = 0; b < TT; ++b) shm[threadIdx.x >> 5][b] = emax[b];
  __syncthreads();
  if (threadIdx.x < TT) {
    int E = -0x7FFFFFFF;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) E = max(E, shm[w][threadIdx.x]);
    if (E == -0x7FFFFFFF) E = 0;  // every coefficient of the column is zero
    if (anybad) E = 0x7FFFFFFF;
    Es[threadIdx.x] = E;
    S.cexp[(size_t)r * TT + threadIdx.x] = E;
  }
  __syncthreads();
  unsigned char* CB = S.CB + (size_t)r * S.maxV * NU * 32;
  // one thread per (vector a, column b): its 20 rows; then the padding rows of every vector
  for (int q = threadIdx.x; q < p * TT; q += blockDim.x) {
    const int a = q / TT, b = q % TT;
    const double2 h = H[q];
    int dre[gst::SL], dim[gst::SL];
    const int E = Es[b];
    const int sh = (E == 0x7FFFFFFF) ? 0x7FFFFFFF : E - vexp[a];
    gst::digits8(sh == 0x7FFFFFFF ? 0.0 : h.x, sh, dre);
    gst::digits8(sh == 0x7FFFFFFF ? 0.0 : h.y, sh, dim);
    unsigned char* img = CB + (size_t)a * NU * 32;
#pragma unroll
    for (int part = 0; part < 2; ++part) {
#pragma unroll
      for (int w = 0; w < 10; ++w) {
        const int n = (2 * b + part) * 10 + w;
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          // G[a, c, (b, part)]: (Re h, -Im h) for part 0, (Im h, Re h) for part 1
          int v[gst::SL];
#pragma unroll
          for (int i = 0; i < gst::SL; ++i) {
            const int j = w - i;
            int dj = 0;
            if (j >= 0 && j < gst::SL) {
              if (part == 0) dj = c == 0 ? dre[j] : -dim[j];
              else dj = c == 0 ? dim[j] : dre[j];
            }
            v[i] = dj;
          }
          *reinterpret_cast<uint4*>(img + gst::ns_off(n, c)) =
              make_uint4(gst::bf16x2(v[0], v[1]), gst::bf16x2(v[2], v[3]), gst::bf16x2(v[4], v[5]),
                         gst::bf16x2(v[6], v[7]));
        }
      }
    }
  }
  for (int q = threadIdx.x; q < p * (NU - 20 * TT) * 2; q += blockDim.x) {
    const int a = q / ((NU - 20 * TT) * 2), rest = q % ((NU - 20 * TT) * 2);
    const int n = 20 * TT + rest / 2, c = rest & 1;
    *reinterpret_cast<uint4*>(CB + (size_t)a * NU * 32 + gst::ns_off(n, c)) = make_uint4(0, 0, 0, 0);
  }
}

}  // namespace

// ------------------------------------------------------------------ tensor-core kernels
namespace {

__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}

// shared-memory matrix descriptor, K-major, no swizzle: 8x8 core matrices (8 rows of 16 bytes),
// cores adjacent in K 128 B apart (leading offset), 8-row groups 256 B apart (stride offset)
__device__ __forceinline__ uint64_t ns_desc(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)(256 >> 4) << 32) |
         ((uint64_t)1 << 46);
}

// K-major, 128-byte swizzle, 8-row groups `sbo` bytes apart
__device__ __forceinline__ uint64_t sw128_desc_sbo(uint32_t saddr, uint32_t sbo) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 1, %0;" ::"n"(gst::EPI_THREADS) : "memory"); }

__device__ __forceinline__ unsigned char* align1024(unsigned char* p) {
  return reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(p) + 1023) & ~(uintptr_t)1023);
}

// H partials of this pass: CTA x of slot r takes stages [s0, s1) of the 2 Dp / 64 (plane, node
// chunk) stages and writes <v_a, w_b> over its nodes to Hpart[((r maxV + a) t + b) GX + x].
template <int TT>
__global__ void __launch_bounds__(gst::THREADS, 1) gst_dot_kernel(KState S, const double2* __restrict__ W, int* err,
                                                                  long long budget) {
  using namespace gst;
  constexpr int N = 16 * TT, BB = dot_bbytes(TT), NCOL = 2 * TT;
  constexpr uint32_t IDESC =
      (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
  const int r = blockIdx.y;
  if (S.done[r]) return;
  const int p = S.nV[r];
  extern __shared__ __align__(16) unsigned char smraw[];
  unsigned char* sm = align1024(smraw);
  unsigned char* sa = sm;
  unsigned char* sb = sa + DOT_NA * ATILE;
  double* acc64 = reinterpret_cast<double*>(sb + DOT_NB * DOT_SC * BB);         // [DOT_MAXT * 16][NCOL]
  long long* isum = reinterpret_cast<long long*>(acc64 + DOT_MAXT * 16 * NCOL);  // [DOT_MAXT * 16][NCOL][2]
  uint64_t* full_a = reinterpret_cast<uint64_t*>(isum + DOT_MAXT * 16 * NCOL * 2);
  uint64_t* empty_a = full_a + DOT_NA;
  uint64_t* full_b = empty_a + DOT_NA;
  uint64_t* empty_b = full_b + DOT_NB;
  uint64_t* accfull = empty_b + DOT_NB;
  uint64_t* accempty = accfull + DOT_MAXT;
  uint64_t* fin = accempty + DOT_MAXT;
  unsigned char** vcache = reinterpret_cast<unsigned char**>(fin + 1);  // [PTR_CACHE]
  __shared__ uint32_t taddr_s;
  __shared__ int abort_s;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int a = threadIdx.x; a < min(p, PTR_CACHE); a += blockDim.x) vcache[a] = S.VSptr[(size_t)r * S.maxV + a];
  if (threadIdx.x == 0) {
    for (int q = 0; q < DOT_NA; ++q) { mbar_init(&full_a[q], 1); mbar_init(&empty_a[q], 1); }
    for (int q = 0; q < DOT_NB; ++q) { mbar_init(&full_b[q], 1); mbar_init(&empty_b[q], 1); }
    for (int q = 0; q < DOT_MAXT; ++q) { mbar_init(&accfull[q], 1); mbar_init(&accempty[q], EPI_THREADS / 32); }
    mbar_init(fin, 1);
    abort_s = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    fence_proxy_async();
  }
  if (warp == 1) {
    tc::tmem_alloc(&taddr_s, 512);
    tc::tmem_relinquish();
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = taddr_s;
  const int NST = S.Dp / (32 * DOT_SC);  // 2 planes x Dp / 64 chunks / DOT_SC
  const int per = (NST + (int)gridDim.x - 1) / (int)gridDim.x;
  const int s0 = min(NST, (int)blockIdx.x * per), s1 = min(NST, s0 + per), ns = s1 - s0;
  const int nT = (p + 15) / 16, rounds = (nT + DOT_MAXT - 1) / DOT_MAXT;
  unsigned char* const* vs = S.VSptr + (size_t)r * S.maxV;

  if (warp == 0) {
    // ---------------------------------------------------------------- producer
    // lane 0 waits for the ring slot and posts the byte count; lane v then issues the copy of
    // vector v of the tile (16 copies in parallel instead of one after another)
    int ka = 0;
    bool ok = true;
    for (int rd = 0; rd < rounds && ok; ++rd) {
      const int T0 = rd * DOT_MAXT, nt = min(DOT_MAXT, nT - T0);
      for (int s = s0; s < s1 && ok; ++s) {
        for (int T = 0; T < nt; ++T) {
          const int slot = ka % DOT_NA;
          const int v0 = (T0 + T) * 16, nv = min(16, p - v0);
          if (lane == 0) {
            if (ka >= DOT_NA && !mbar_wait(&empty_a[slot], ((unsigned)(ka / DOT_NA) & 1u) ^ 1u, err, budget)) ok = false;
            if (tc::aborted(&abort_s)) ok = false;
            if (ok) mbar_expect_tx(&full_a[slot], nv * DOT_SC * 1024);
          }
          ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
          if (!ok) break;
          if (lane < nv) {
            const unsigned char* img = v0 + lane < PTR_CACHE ? vcache[v0 + lane] : vs[v0 + lane];
            bulk_g2s(sa + slot * ATILE + lane * DOT_SC * 1024, img + (size_t)s * DOT_SC * 1024, DOT_SC * 1024,
                     &full_a[slot]);
          }
          ++ka;
        }
      }
    }
    if (!ok && lane == 0) {
      *(volatile int*)&abort_s = 1;
      // let the copies in flight land before the CTA leaves
      for (int k = max(0, ka - DOT_NA); k < ka; ++k)
        mbar_wait(&full_a[k % DOT_NA], (unsigned)(k / DOT_NA) & 1u, err, budget);
    }
  } else if (warp == 1) {
    // ---------------------------------------------------------------- MMA issuer
    if (lane == 0) {
      int ka = 0, kb = 0;
      int cnt[DOT_MAXT];
      for (int T = 0; T < DOT_MAXT; ++T) cnt[T] = 0;
      bool ok = true;
      for (int rd = 0; rd < rounds && ok; ++rd) {
        const int T0 = rd * DOT_MAXT, nt = min(DOT_MAXT, nT - T0);
        for (int si = 0; si < ns && ok; ++si) {
          const int bslot = kb % DOT_NB;
          if (!mbar_wait(&full_b[bslot], (unsigned)(kb / DOT_NB) & 1u, err, budget)) { ok = false; break; }
          const bool pstart = (si % DOT_FL) == 0, pend = (si % DOT_FL) == DOT_FL - 1 || si == ns - 1;
          for (int T = 0; T < nt; ++T) {
            const int slot = ka % DOT_NA;
            if (!mbar_wait(&full_a[slot], (unsigned)(ka / DOT_NA) & 1u, err, budget)) { ok = false; break; }
            if (pstart && cnt[T] > 0 && !mbar_wait(&accempty[T], (unsigned)(cnt[T] - 1) & 1u, err, budget)) {
              ok = false;
              break;
            }
            if (tc::aborted(&abort_s)) { ok = false; break; }
            tc::fence_after();
            // A: vector v's DOT_SC 1 KB atoms at v DOT_SC KB (8-row groups DOT_SC KB apart);
            // B: the stage's DOT_SC blocks of the new columns' digits one after the other
            const uint32_t a0 = smem_u32(sa + slot * ATILE), b0 = smem_u32(sb + bslot * DOT_SC * BB);
#pragma unroll
            for (int k = 0; k < DOT_SC; ++k)
#pragma unroll
              for (int kk = 0; kk < 4; ++kk)
                mma_bf16(tmem + T * N, sw128_desc_sbo(a0 + k * 1024 + kk * 32, DOT_SC * 1024),
                         tc::sw128_desc(b0 + k * BB + kk * 32), IDESC, (pstart && k == 0 && kk == 0) ? 0u : 1u);
            tc::commit(&empty_a[slot]);
            ++ka;
            if (pend) {
              tc::commit(&accfull[T]);
              ++cnt[T];
            }
          }
          if (!ok) break;
          tc::commit(&empty_b[bslot]);
          ++kb;
        }
      }
      if (!ok) *(volatile int*)&abort_s = 1;
      tc::commit(fin);  // arrives once every MMA issued above has completed
      mbar_wait(fin, 0, err, budget);
    }
  } else if (warp < 2 + EPI_THREADS / 32) {
    // ---------------------------------------------------------------- epilogue
    // Exact integer accumulation: a flush holds, in this thread's lane (vector a, digit i), the
    // sums acc_j (|acc_j| < 2^24, exact in FP32) for every column b' and digit j.  They are
    // combined in int64: H = sum over i + j <= 4 of acc_j 2^{7 (4 - i - j)} and L = sum over
    // 5 <= i + j <= 9 of acc_j 2^{7 (9 - i - j)} (each below 2^52.1; digit pairs of weight
    // 2^-70 of the leading pair and below are dropped); the eight digit rows of a vector are
    // summed by shuffles (below 2^55.1) and lane i = 0 adds them into the CTA's int64 sums,
    // converted to FP64 (value H 2^-42 + L 2^-77 in units of 2^{e_a + f_b}) every DOT_CONV
    // flushes and at the end.  No FP64 arithmetic per flush.
    const int wq = warp & 3, et = threadIdx.x - 64;
    const int R = wq * 32 + lane, i = R & 7, vloc = R >> 3;
    const uint32_t tlane = tmem + ((uint32_t)(wq * 32) << 16);
    int cnt[DOT_MAXT];
    for (int T = 0; T < DOT_MAXT; ++T) cnt[T] = 0;
    bool ok = true;
    auto convert = [&](int nt) {
      if (i != 0) return;
      for (int T = 0; T < nt; ++T) {
        long long* is = isum + (size_t)(T * 16 + vloc) * NCOL * 2;
        double* dst = acc64 + (size_t)(T * 16 + vloc) * NCOL;
#pragma unroll
        for (int b = 0; b < NCOL; ++b) {
          dst[b] += ldexp((double)is[2 * b], -42) + ldexp((double)is[2 * b + 1], -77);
          is[2 * b] = 0;
          is[2 * b + 1] = 0;
        }
      }
    };
    for (int rd = 0; rd < rounds; ++rd) {
      const int T0 = rd * DOT_MAXT, nt = min(DOT_MAXT, nT - T0);
      for (int e = et; e < DOT_MAXT * 16 * NCOL; e += EPI_THREADS) {
        acc64[e] = 0;
        isum[2 * e] = 0;
        isum[2 * e + 1] = 0;
      }
      epi_sync();
      const int nflush = (ns + DOT_FL - 1) / DOT_FL;
      for (int f = 0; f < nflush && ok; ++f) {
        for (int T = 0; T < nt; ++T) {
          // warp-uniform decision: the shuffles below need every lane of the warp
          const bool got = mbar_wait(&accfull[T], (unsigned)cnt[T] & 1u, err, budget) && !tc::aborted(&abort_s);
          if (!__all_sync(0xffffffffu, got)) {
            ok = false;
            break;
          }
          ++cnt[T];
          tc::fence_after();
          uint32_t u[(N + 31) / 32 * 32];
#pragma unroll
          for (int q = 0; q < (N + 31) / 32; ++q) {
            uint32_t (&uq)[32] = *reinterpret_cast<uint32_t(*)[32]>(&u[32 * q]);
            tc::tmem_ld32(tlane + T * N + 32 * q, uq);
          }
          tc::tmem_wait_ld();
          tc::fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(&accempty[T]);
          long long hs[NCOL], ls[NCOL];
#pragma unroll
          for (int b = 0; b < NCOL; ++b) {
            long long h = 0, l = 0;
#pragma unroll
            for (int j = 0; j < SL; ++j) {
              const long long x = gst::f2i_exact(__uint_as_float(u[b * SL + j]));
              const int sh = 4 - i - j, sl = 9 - i - j;
              if (sh >= 0) h += x * (1ll << (7 * sh));
              else if (sl >= 0) l += x * (1ll << (7 * sl));
            }
#pragma unroll
            for (int o = 1; o < 8; o <<= 1) {
              h += __shfl_xor_sync(0xffffffffu, h, o);
              l += __shfl_xor_sync(0xffffffffu, l, o);
            }
            hs[b] = h;
            ls[b] = l;
          }
          if (i == 0) {
            long long* is = isum + (size_t)(T * 16 + vloc) * NCOL * 2;
#pragma unroll
            for (int b = 0; b < NCOL; ++b) {
              is[2 * b] += hs[b];
              is[2 * b + 1] += ls[b];
            }
          }
        }
        if ((f + 1) % DOT_CONV == 0) convert(nt);
      }
      convert(nt);
      epi_sync();
      for (int e = et; e < nt * 16 * TT; e += EPI_THREADS) {
        const int vl = e / TT, b = e % TT, a = T0 * 16 + vl;
        if (a >= p) continue;
        const int ea = S.vexp[(size_t)r * S.maxV + a];
        const int fb = frexp_exp_bits(S.wmaxb[(size_t)r * TT + b]);
        double2 h;
        if (ea == 0x7FFFFFFF || fb == 0x7FFFFFFF) {
          h = make_double2(__longlong_as_double(0x7FF8000000000000ll), __longlong_as_double(0x7FF8000000000000ll));
        } else {
          h = make_double2(ldexp(acc64[vl * NCOL + 2 * b], ea + fb), ldexp(acc64[vl * NCOL + 2 * b + 1], ea + fb));
        }
        S.Hpart[((size_t)(r * S.maxV + a) * TT + b) * S.GX + blockIdx.x] = h;
      }
      epi_sync();
    }
  } else {
    // ---------------------------------------------------------------- slicer
    // The B operand of every stage (plane c, the 128 nodes from g0), formed here from W instead
    // of a stored image: thread i takes node g0 + i and, for every new column b, the eight
    // digits of Re w_b and Im w_b relative to 2^{f_b} (f_b from the column maxima); plane 0
    // gives rows (2b, j) = Re, (2b + 1, j) = Im, plane 1 rows (2b, j) = Im, (2b + 1, j) = -Re,
    // 128-byte swizzled as the MMA reads them.  The next stage's entries of W are requested
    // before this stage is sliced.
    const int i = threadIdx.x - (2 + EPI_THREADS / 32) * 32;
    const int kk = i & 63, qq = i >> 6;
    const int chunks = S.Dp / 64;  // a multiple of DOT_SC: no stage straddles the two planes
    const size_t D = S.D;
    const double2* Wr = W + (size_t)r * TT * D;
    int fe[TT];
#pragma unroll
    for (int b = 0; b < TT; ++b) fe[b] = frexp_exp_bits(S.wmaxb[(size_t)r * TT + b]);
    auto fetch = [&](int s, double2 (&w)[TT]) {
      const size_t g = (size_t)((s * DOT_SC) % chunks) * 64 + i;
#pragma unroll
      for (int b = 0; b < TT; ++b) w[b] = (g < D && fe[b] != 0x7FFFFFFF) ? Wr[b * D + g] : make_double2(0, 0);
    };
    double2 cur[TT], nxt[TT];
    if (ns > 0) fetch(s0, cur);
    int kb = 0;
    bool stop = false;
    for (int rd = 0; rd < rounds && !stop; ++rd) {
      for (int s = s0; s < s1; ++s) {
        fetch(s + 1 < s1 ? s + 1 : s0, nxt);  // after the last stage: the next round's first
        const int slot = kb % DOT_NB;
        const int bad =
            ((kb >= DOT_NB && !mbar_wait(&empty_b[slot], ((unsigned)(kb / DOT_NB) & 1u) ^ 1u, err, budget)) ||
             tc::aborted(&abort_s))
                ? 1
                : 0;
        // the slicers decide together, so that all of them meet at the barrier below
        int any_bad;
        asm volatile(
            "{\n .reg .pred p, q;\n setp.ne.u32 q, %1, 0;\n bar.red.or.pred p, 2, %2, q;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(any_bad)
            : "r"(bad), "n"(SLICE_THREADS)
            : "memory");
        if (any_bad) {
          *(volatile int*)&abort_s = 1;
          stop = true;
          break;
        }
        const bool im_plane = (s * DOT_SC) / chunks != 0;
        unsigned char* blk = sb + slot * DOT_SC * BB + qq * BB;
#pragma unroll
        for (int b = 0; b < TT; ++b) {
          int dr[SL], di[SL];
          digits8(cur[b].x, fe[b], dr);
          digits8(cur[b].y, fe[b], di);
#pragma unroll
          for (int j = 0; j < SL; ++j) {
            const int n0 = (2 * b) * 8 + j, n1 = n0 + 8;
            const int col = (((kk >> 3) ^ j) << 4) + (kk & 7) * 2;
            const int v0 = im_plane ? di[j] : dr[j], v1 = im_plane ? -dr[j] : di[j];
            *reinterpret_cast<__nv_bfloat16*>(blk + n0 * 128 + col) = __float2bfloat16_rn((float)v0);
            *reinterpret_cast<__nv_bfloat16*>(blk + n1 * 128 + col) = __float2bfloat16_rn((float)v1);
          }
        }
        fence_proxy_async_smem();  // the tensor cores read the tile through the async proxy
        asm volatile("bar.sync 2, %0;" ::"n"(SLICE_THREADS) : "memory");
        if (i == 0) mbar_arrive(&full_b[slot]);
        ++kb;
#pragma unroll
        for (int b = 0; b < TT; ++b) cur[b] = nxt[b];
      }
    }
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 1) tc::tmem_dealloc(tmem, 512);
}

// W_b -= sum_a v_a h_ab for the new columns of slot r: tiles of 384 nodes (grid-stride over the
// slot's Dp / 384 tiles); per basis vector one stage = the three 128-node images of NI and the
// coefficient image CB, three MMAs (M = 128 nodes, N = NU, K = 16) into one of two tensor-memory
// buffers; every 64 vectors the buffer is read out and its weight groups summed in int64.
template <int TT>
__global__ void __launch_bounds__(gst::UPD_THREADS, 1) gst_upd_kernel(KState S, double2* __restrict__ W,
                                                                      int track_max, int* err, long long budget) {
  using namespace gst;
  constexpr int NU = nu_rows(TT), CBB = NU * 32, STB = upd_stage_bytes(TT), NOUT = 2 * TT, NCOLS = 20 * TT;
  constexpr uint32_t IDESC =
      (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(NU >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
  const int r = blockIdx.y;
  if (S.done[r]) return;
  const int p = S.nV[r];
  extern __shared__ __align__(16) unsigned char smraw[];
  unsigned char* sm = align1024(smraw);
  uint64_t* full = reinterpret_cast<uint64_t*>(sm + UPD_NS * STB);
  uint64_t* empty = full + UPD_NS;
  uint64_t* accfull = empty + UPD_NS;
  uint64_t* accempty = accfull + 2;
  uint64_t* fin = accempty + 2;
  unsigned char** vcache = reinterpret_cast<unsigned char**>(fin + 1);  // [PTR_CACHE]
  __shared__ uint32_t taddr_s;
  __shared__ int abort_s;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int a = threadIdx.x; a < min(p, PTR_CACHE); a += blockDim.x) vcache[a] = S.VSptr[(size_t)r * S.maxV + a];
  if (threadIdx.x == 0) {
    for (int q = 0; q < UPD_NS; ++q) { mbar_init(&full[q], 1); mbar_init(&empty[q], 1); }
    for (int q = 0; q < 2; ++q) { mbar_init(&accfull[q], 1); mbar_init(&accempty[q], (UPD_THREADS - 64) / 32); }
    mbar_init(fin, 1);
    abort_s = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    fence_proxy_async();
  }
  if (warp == 1) {
    tc::tmem_alloc(&taddr_s, 512);
    tc::tmem_relinquish();
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = taddr_s;
  const int ntile = S.Dp / UPD_NODES;
  const int nseg = (p + UPD_SEG - 1) / UPD_SEG;
  unsigned char* const* vs = S.VSptr + (size_t)r * S.maxV;
  const unsigned char* CB = S.CB + (size_t)r * S.maxV * CBB;
  const size_t ni_off = (size_t)32 * S.Dp;

  if (warp == 0) {
    // ---------------------------------------------------------------- producer
    if (lane == 0) {
      int k = 0;
      bool ok = true;
      for (int tile = blockIdx.x; tile < ntile && ok; tile += gridDim.x) {
        for (int a = 0; a < p; ++a) {
          const int slot = k % UPD_NS;
          if (k >= UPD_NS && !mbar_wait(&empty[slot], ((unsigned)(k / UPD_NS) & 1u) ^ 1u, err, budget)) {
            ok = false;
            break;
          }
          if (tc::aborted(&abort_s)) { ok = false; break; }
          unsigned char* st = sm + slot * STB;
          const unsigned char* ni =
              (a < PTR_CACHE ? vcache[a] : vs[a]) + ni_off + (size_t)(UPD_PARTS * tile) * 4096;
          mbar_expect_tx(&full[slot], 4096 * UPD_PARTS + CBB);
          bulk_g2s(st, ni, 4096 * UPD_PARTS, &full[slot]);  // the tile's 128-node images are adjacent
          bulk_g2s(st + 4096 * UPD_PARTS, CB + (size_t)a * CBB, CBB, &full[slot]);
          ++k;
        }
      }
      if (!ok) {
        *(volatile int*)&abort_s = 1;
        for (int q = max(0, k - UPD_NS); q < k; ++q)
          mbar_wait(&full[q % UPD_NS], (unsigned)(q / UPD_NS) & 1u, err, budget);
      }
    }
  } else if (warp == 1) {
    // ---------------------------------------------------------------- MMA issuer
    if (lane == 0) {
      int k = 0, sc = 0;
      bool ok = true;
      for (int tile = blockIdx.x; tile < ntile && ok; tile += gridDim.x) {
        for (int sg = 0; sg < nseg && ok; ++sg) {
          const int buf = sc & 1;
          if (sc >= 2 && !mbar_wait(&accempty[buf], (unsigned)((sc >> 1) - 1) & 1u, err, budget)) {
            ok = false;
            break;
          }
          const int a0 = sg * UPD_SEG, a1 = min(p, a0 + UPD_SEG);
          for (int a = a0; a < a1; ++a) {
            const int slot = k % UPD_NS;
            if (!mbar_wait(&full[slot], (unsigned)(k / UPD_NS) & 1u, err, budget) || tc::aborted(&abort_s)) {
              ok = false;
              break;
            }
            tc::fence_after();
            const uint32_t st = smem_u32(sm + slot * STB);
            const uint64_t bdesc = ns_desc(st + 4096 * UPD_PARTS);
#pragma unroll
            for (int h = 0; h < UPD_PARTS; ++h)
              mma_bf16(tmem + (buf * UPD_PARTS + h) * NU, ns_desc(st + h * 4096), bdesc, IDESC, a > a0 ? 1u : 0u);
            tc::commit(&empty[slot]);
            ++k;
          }
          if (!ok) break;
          tc::commit(&accfull[buf]);
          ++sc;
        }
      }
      if (!ok) *(volatile int*)&abort_s = 1;
      tc::commit(fin);
      mbar_wait(fin, 0, err, budget);
    }
  } else {
    // ---------------------------------------------------------------- epilogue
    // A buffer holds, for this thread's node and column b', the sums acc_w of weight group w
    // (|acc_w| < 2^24, exact in FP32).  They are combined exactly in int64: H = sum_{w <= 4}
    // acc_w 2^{7 (4 - w)}, L = sum_{5 <= w <= 9} acc_w 2^{7 (9 - w)} (each below 2^52.1 per
    // segment), summed over the segments, and converted once per tile: the value is
    // H 2^{E - 42} + L 2^{E - 77}.
    const int wq = warp & 3, h = (warp - 2) >> 2;  // node part of this warp
    const int R = wq * 32 + lane;
    const uint32_t tlane = tmem + ((uint32_t)(wq * 32) << 16);
    int Es[TT];
    bool nan_out = false;
#pragma unroll
    for (int b = 0; b < TT; ++b) {
      Es[b] = S.cexp[(size_t)r * TT + b];
      nan_out |= Es[b] == 0x7FFFFFFF;
    }
    const size_t D = S.D;
    double2* Wr = W + (size_t)r * TT * D;
    int sc = 0;
    bool ok = true;
    for (int tile = blockIdx.x; tile < ntile && ok; tile += gridDim.x) {
      long long oh[NOUT], ol[NOUT];
#pragma unroll
      for (int b = 0; b < NOUT; ++b) oh[b] = ol[b] = 0;
      for (int sg = 0; sg < nseg; ++sg) {
        const int buf = sc & 1;
        const bool got = mbar_wait(&accfull[buf], (unsigned)(sc >> 1) & 1u, err, budget) && !tc::aborted(&abort_s);
        if (!__all_sync(0xffffffffu, got)) {  // warp-uniform: the warp reductions need every lane
          ok = false;
          break;
        }
        ++sc;
        tc::fence_after();
#pragma unroll
        for (int q = 0; q < (NCOLS + 31) / 32; ++q) {
          uint32_t u[32];
          tc::tmem_ld32(tlane + (buf * UPD_PARTS + h) * NU + 32 * q, u);
          tc::tmem_wait_ld();
#pragma unroll
          for (int c = 0; c < 32; ++c) {
            const int col = 32 * q + c, b = col / 10, w = col % 10;
            if (col >= NCOLS) break;
            const long long x = gst::f2i_exact(__uint_as_float(u[c]));
            if (w <= 4) oh[b] += x * (1ll << (7 * (4 - w)));
            else ol[b] += x * (1ll << (7 * (9 - w)));
          }
        }
        tc::fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&accempty[buf]);
      }
      if (!ok) break;
      const size_t g = (size_t)tile * UPD_NODES + h * 128 + R;
      unsigned long long mx[TT];
#pragma unroll
      for (int b = 0; b < TT; ++b) mx[b] = 0;
      if (g < D) {
#pragma unroll
        for (int b = 0; b < TT; ++b) {
          double2 w = Wr[b * D + g];
          if (nan_out) {
            w.x = w.y = __longlong_as_double(0x7FF8000000000000ll);
          } else {
            // H 2^{E-42} + L 2^{E-77}: H alone resolves 2^{E-42} only, coarser than the FP64
            // rounding of values below 2^{E+11}, so both parts are converted and added in FP64
            const int Eb = Es[b];
            w.x -= i64_scaled(oh[2 * b], Eb - 42) + i64_scaled(ol[2 * b], Eb - 77);
            w.y -= i64_scaled(oh[2 * b + 1], Eb - 42) + i64_scaled(ol[2 * b + 1], Eb - 77);
          }
          Wr[b * D + g] = w;
          mx[b] = max(gst::abs_bits(w.x), gst::abs_bits(w.y));
        }
      }
      if (track_max) {
        // the next pass's column maxima (its slice scale), instead of another pass over W
#pragma unroll
        for (int b = 0; b < TT; ++b) {
          const unsigned long long mw = warp_max_u64(mx[b]);
          if (lane == 0 && mw) atomicMax(&S.wmaxb[(size_t)r * TT + b], mw);
        }
      }
    }
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 1) tc::tmem_dealloc(tmem, 512);
}

}  // namespace

// ------------------------------------------------------------------ host side
template <int TT>
static cudaError_t set_attrs_t() {
  cudaError_t e = cudaFuncSetAttribute((const void*)gst_dot_kernel<TT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)gst::dot_smem(TT));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute((const void*)gst_upd_kernel<TT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)gst::upd_smem(TT));
  return e;
}

cudaError_t gst_set_attributes(int t) {
  static_assert(gst::dot_smem(4) <= 232448 && gst::upd_smem(4) <= 232448, "shared memory");
  // the last part of buffer 1 is read in 32-column loads
  static_assert((2 * gst::UPD_PARTS - 1) * gst::nu_rows(4) + 96 <= 512, "tensor memory of the update");
  switch (t) {
    case 1: return set_attrs_t<1>();
    case 2: return set_attrs_t<2>();
    case 3: return set_attrs_t<3>();
    default: return set_attrs_t<4>();
  }
}

// Slice images of the basis vectors [vnew0, vnew1) of every slot (mode 1: only the slots being
// admitted).  Launches: a memset and two kernels.
void gst_slice_basis(Engine& E, const KState& K, int S, int mode) {
  cudaMemsetAsync(K.vmaxb, 0, sizeof(unsigned long long) * S * K.t, E.stream);
  const int gx = std::max(1, std::min(E.num_sms * 2 / std::max(1, S), (K.D + 255) / 256));
  gst_vscan_kernel<<<dim3(gx, S, K.t), 256, 0, E.stream>>>(K, mode);
  const int gs = std::max(1, std::min(E.num_sms * 4 / std::max(1, S), K.Dp / 256));
  gst_vslice_kernel<<<dim3(gs, S, K.t), 256, 0, E.stream>>>(K, mode);
  E.count_launch(2);
}

template <int TT>
static void prep_w_t(Engine& E, const KState& K, int S, const double2* W, bool first) {
  if (first) {  // later passes take the column maxima from the previous pass's update
    cudaMemsetAsync(K.wmaxb, 0, sizeof(unsigned long long) * S * TT, E.stream);
    gst_wscan_kernel<TT><<<dim3(K.GX, S), 256, 0, E.stream>>>(K, W, 1);
    E.count_launch(1);
  }
}
template <int TT>
static void dot_t(Engine& E, const KState& K, int S, const double2* W, int gd) {
  gst_dot_kernel<TT><<<dim3(gd, S), gst::THREADS, gst::dot_smem(TT), E.stream>>>(K, W, E.err, E.opts.timeout_cycles);
  E.count_launch(1);
}

template <int TT>
static void pass_b_t(Engine& E, const KState& K, int S, double2* W, int gu, bool track_max) {
  gst_cslice_kernel<TT><<<S, 256, 0, E.stream>>>(K);
  if (track_max) cudaMemsetAsync(K.wmaxb, 0, sizeof(unsigned long long) * S * TT, E.stream);
  gst_upd_kernel<TT><<<dim3(gu, S), gst::UPD_THREADS, gst::upd_smem(TT), E.stream>>>(K, W, track_max ? 1 : 0, E.err,
                                                                                    E.opts.timeout_cycles);
  E.count_launch(2);
}

// CTAs per slot of the inner-product kernel (at most K.GX: the stride of the partials)
int gst_dot_ctas(const Engine& E, const KState& K, int S) {
  return std::max(1, std::min({E.num_sms / std::max(1, S), K.GX, K.Dp / 32}));
}
int gst_upd_ctas(const Engine& E, const KState& K, int S) {
  return std::max(1, std::min(E.num_sms / std::max(1, S), K.Dp / gst::UPD_NODES));
}

// First part of a Gram-Schmidt pass (the first pass only): the new columns' maxima and the
// deflation reference.
void gst_prepare_columns(Engine& E, const KState& K, int S, const double2* W, bool first) {
  switch (K.t) {
    case 1: prep_w_t<1>(E, K, S, W, first); break;
    case 2: prep_w_t<2>(E, K, S, W, first); break;
    case 3: prep_w_t<3>(E, K, S, W, first); break;
    default: prep_w_t<4>(E, K, S, W, first); break;
  }
}

// Second part: the inner-product partials (gst_dot_ctas CTAs per slot), the new columns sliced
// from W inside the kernel.
void gst_inner_products(Engine& E, const KState& K, int S, const double2* W) {
  const int gd = gst_dot_ctas(E, K, S);
  switch (K.t) {
    case 1: dot_t<1>(E, K, S, W, gd); break;
    case 2: dot_t<2>(E, K, S, W, gd); break;
    case 3: dot_t<3>(E, K, S, W, gd); break;
    default: dot_t<4>(E, K, S, W, gd); break;
  }
}

// Last part, after the partials are summed into Hthis: the coefficient images and the update.
void gst_pass_update(Engine& E, const KState& K, int S, double2* W, bool track_max) {
  const int gu = gst_upd_ctas(E, K, S);
  switch (K.t) {
    case 1: pass_b_t<1>(E, K, S, W, gu, track_max); break;
    case 2: pass_b_t<2>(E, K, S, W, gu, track_max); break;
    case 3: pass_b_t<3>(E, K, S, W, gu, track_max); break;
    default: pass_b_t<4>(E, K, S, W, gu, track_max); break;
  }
}

// bytes of the slice images of one basis vector, of a slot's coefficient images
size_t gst_vector_bytes(size_t Dp) { return 64 * Dp; }
size_t gst_cimage_bytes(int maxV, int t) { return (size_t)maxV * gst::nu_rows(t) * 32; }
int gst_nu_rows(int t) { return gst::nu_rows(t); }

}  // namespace hh
