// hh_apply_preconditioner_noalloc: the preconditioner apply (one directional sweep) for
// callers that cannot allocate device memory while they run -- for example code that runs
// under a fixed device-memory budget taken at start-up, host frameworks whose caching
// allocator owns every byte of the device, or real-time paths that must not pay for
// cudaMalloc / cudaFree (which can synchronise the whole device).  The kernels are the
// same as hh_apply_preconditioner's; only their scratch moves: the packed input, the
// sweep output, the correction array, the interface arrays, the column tables and the split-K
// slices live in one
// file-scope device array of fixed size.  The array is reserved on a device when this file's
// module is loaded there, which CUDA's lazy module loading does at the first use of one of its
// symbols; hh_setup makes that use (it resolves the array's device address), so the array is
// reserved on the handle's device before any call of this entry point, and held until the
// process exits.
//
// Scratch contents: nothing in the array has to start at zero.  Each call rewrites the
// whole packed input (padding entries included) and the column tables, and every sweep step
// writes the lines it produces before a later step reads them.  The array keeps whatever
// the last call left in it.
//
// Sharing: all calls in the process share the one array per device.  Calls whose GPU
// work overlaps (two handles on different streams, two threads) race on it; callers must
// serialise them.
#include <cstdio>
#include <mutex>
#include <string>

#include "common.cuh"
#include "engine.h"

namespace hh {

void launch_pack(Engine& E, const double2* const* srcptr, const double* scale, int C, int t, int4 codes, void* X);
void launch_unpack(Engine& E, const void* X, int C, int t, int4 codes, double2* dst, size_t stride);

// Fixed scratch of the no-allocation entry point: 32 MiB per device.
constexpr size_t kNoAllocScratchBytes = 32ull << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Device address of g_noalloc_scratch for each device, resolved once per device (with that
// device current) by the first hh_setup on it.
constexpr int kMaxDevices = 64;
static std::mutex g_noalloc_mu;
static void* g_noalloc_addr[kMaxDevices] = {};

int noalloc_scratch_address(int device, void** out) {
  if (device < 0 || device >= kMaxDevices) {
    set_error("device index out of range for the no-allocation scratch");
    return HH_EINVAL;
  }
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_addr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      set_error(std::string("cudaGetSymbolAddress of the no-allocation scratch failed: ") + cudaGetErrorString(e));
      return HH_ECUDA;
    }
    g_noalloc_addr[device] = p;
  }
  *out = g_noalloc_addr[device];
  return HH_OK;
}

// column tables of the pack kernel: input column c starts at r + c * D, unscaled
__global__ void noalloc_tables_kernel(const double2* r, size_t D, int ncols, const double2** srcptr, double* scale) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ncols; c += gridDim.x * blockDim.x) {
    srcptr[c] = r + (size_t)c * D;
    scale[c] = 1.0;
  }
}

static size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

static bool is_device_pointer(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

int Engine::apply_preconditioner_noalloc(int dcode, int ncols, const double2* r, double2* z, bool single) {
  const size_t D = (size_t)m * m;
  const size_t arr = sweep_ws_bytes(ncols);
  const size_t off_v = align256(arr);
  const size_t off_w = off_v + align256(arr);
  const size_t off_ptr = off_w + align256(arr);
  const size_t off_scale = off_ptr + align256(sizeof(void*) * ncols);
  const size_t tline = (size_t)m * N * ncols * sweep_elem();  // one-line interface arrays
  const size_t off_t0 = off_scale + align256(sizeof(double) * ncols);
  const size_t off_t1 = off_t0 + align256(tline);
  const size_t need = off_t1 + align256(tline);
  // whatever is left of the array holds split-K slices of the GEMM steps (fewer slices, or
  // none, when it is small)
  const size_t off_part = need;
  if (need > kNoAllocScratchBytes) {
    set_error("hh_apply_preconditioner_noalloc: this grid and column count need " + std::to_string(need) +
              " bytes of scratch, more than its fixed " + std::to_string(kNoAllocScratchBytes) + " bytes");
    return HH_EINVAL;
  }
  void* base = nullptr;
  int rc = noalloc_scratch_address(device, &base);
  if (rc) return rc;
  unsigned char* s = reinterpret_cast<unsigned char*>(base);
  void* rin = s;
  void* v = s + off_v;
  void* w = s + off_w;
  const double2** tab = reinterpret_cast<const double2**>(s + off_ptr);
  double* scale = reinterpret_cast<double*>(s + off_scale);
  noalloc_tables_kernel<<<1, 256, 0, stream>>>(r, D, ncols, tab, scale);
  count_launch();
  int4 codes = make_int4(dcode, dcode, dcode, dcode);
  launch_pack(*this, tab, scale, ncols, 1, codes, rin);
  const size_t part_bytes = kNoAllocScratchBytes > off_part ? kNoAllocScratchBytes - off_part : 0;
  no_alloc_call = true;
  rc = run_sweep_untimed(rin, v, w, ncols, single, part_bytes ? s + off_part : nullptr, part_bytes, false, s + off_t0,
                         s + off_t1);
  no_alloc_call = false;
  if (rc == HH_OK) launch_unpack(*this, v, ncols, 1, codes, z, D);
  cudaError_t e = cudaStreamSynchronize(stream);
  if (rc) return rc;
  if (e != cudaSuccess) {
    set_cuda_error(e, "hh_apply_preconditioner_noalloc");
    return HH_ECUDA;
  }
  return check_device_error("sweep");
}

}  // namespace hh

using namespace hh;

struct hh_handle {
  Engine* E;
};

extern "C" hh_status hh_apply_preconditioner_noalloc(hh_handle* h, uint32_t dir, int ncols, const double* r,
                                                     double* z) {
  if (!h || !r || !z || ncols < 1) return (set_error("bad arguments"), HH_EINVAL);
  int code;
  switch (dir) {
    case HH_DIR_LR: code = DC_LR; break;
    case HH_DIR_RL: code = DC_RL; break;
    case HH_DIR_BT: code = DC_BT; break;
    case HH_DIR_TB: code = DC_TB; break;
    default: return (set_error("dir must be exactly one HH_DIR_* bit"), HH_EINVAL);
  }
  Engine& E = *h->E;
  if (E.fd) return (set_error("the no-allocation entry point serves the P1 mode only"), HH_EINVAL);
  std::lock_guard<std::mutex> lk(E.solve_mu);
  cudaSetDevice(E.device);
  if (!is_device_pointer(r) || !is_device_pointer(z))
    return (set_error("hh_apply_preconditioner_noalloc takes device pointers only (host buffers would need staging)"),
            HH_EINVAL);
  return (hh_status)E.apply_preconditioner_noalloc(code, ncols, (const double2*)r, (double2*)z,
                                                   E.opts.single_sweep != 0);
}
