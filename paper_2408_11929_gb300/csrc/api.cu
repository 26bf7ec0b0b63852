// C ABI (include/hh.h) on top of the engine: validation, host/device buffer handling,
// timing, statistics and the asynchronous request loop behind hh_submit / hh_poll.
#include <algorithm>
#include <chrono>
#include <memory>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <unordered_map>
#include <vector>

#include "common.cuh"
#include "engine.h"

namespace hh {

static thread_local std::string g_last_error;
void set_error(const std::string& msg) { g_last_error = msg; }

int qr_blocks_per_sm();
int noalloc_scratch_address(int device, void** out);

// ------------------------------------------------------------------ engine helpers
int Engine::dmalloc(void** p, size_t nbytes) {
  *p = nullptr;
  cudaError_t e = cudaMalloc(p, std::max<size_t>(nbytes, 16));
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    set_error(std::string("cudaMalloc of ") + std::to_string(nbytes) + " bytes failed: " + cudaGetErrorString(e));
    return HH_ENOMEM;
  }
  bytes_allocated += nbytes;
  return HH_OK;
}

void Engine::dfree(void* p) {
  if (p) cudaFree(p);
}

unsigned Engine::grid_for(size_t work, int threads) const {
  size_t g = (work + threads - 1) / threads;
  const size_t cap = (size_t)num_sms * 16;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (unsigned)g;
}

cudaError_t Engine::launch_coop(const void* fn, int grid, int block, size_t smem, void** args, int grid_y) {
  count_launch();
  return cudaLaunchCooperativeKernel(fn, dim3(grid, grid_y), dim3(block), args, smem, stream);
}

void Engine::set_cuda_error(cudaError_t e, const char* where) {
  set_error(std::string(where) + ": " + cudaGetErrorString(e));
}

int Engine::check_device_error(const char* where) {
  int h = 0;
  cudaError_t e = cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) {
    set_cuda_error(e, where);
    return HH_ECUDA;
  }
  if (h == DEV_OK) return HH_OK;
  cudaMemsetAsync(err, 0, sizeof(int), stream);
  cudaStreamSynchronize(stream);
  if (h == DEV_TIMEOUT) {
    set_error(std::string(where) + ": a bounded device-side wait ran out of its cycle budget");
    return HH_ETIMEOUT;
  }
  if (h == DEV_SINGULAR) {
    set_error(std::string(where) + ": zero pivot in a strip block inversion");
    return HH_EBREAKDOWN;
  }
  set_error(std::string(where) + ": device error " + std::to_string(h));
  return HH_ENAN;
}

void Engine::tick_begin(int cls) {
  if (!opts.profile) return;
  Tick tk;
  if (event_pool.size() >= 2) {
    tk.a = event_pool.back(); event_pool.pop_back();
    tk.b = event_pool.back(); event_pool.pop_back();
  } else {
    cudaEventCreate(&tk.a);
    cudaEventCreate(&tk.b);
  }
  tk.cls = cls;
  cudaEventRecord(tk.a, stream);
  cur_tick[cls] = tk;
  tick_open[cls] = true;
}

void Engine::tick_end(int cls, double nbytes, double nflops) {
  launches[cls] += 1;
  bytes[cls] += nbytes;
  flops[cls] += nflops;
  if (!opts.profile || !tick_open[cls]) return;
  Tick tk = cur_tick[cls];
  cudaEventRecord(tk.b, stream);
  tk.bytes = nbytes;
  tk.flops = nflops;
  pending_ticks.push_back(tk);
  tick_open[cls] = false;
}

void Engine::collect_ticks() {
  for (auto& tk : pending_ticks) {
    cudaEventSynchronize(tk.b);
    float t = 0;
    if (cudaEventElapsedTime(&t, tk.a, tk.b) == cudaSuccess) ms[tk.cls] += t;
    event_pool.push_back(tk.a);
    event_pool.push_back(tk.b);
  }
  pending_ticks.clear();
}

// ------------------------------------------------------------------ init / teardown
int Engine::init(double k_, int n_, int strips, uint32_t dirs, const hh_opts* o) {
  hh_default_opts(&opts);
  if (o) opts = *o;
  if (!(k_ > 0) || !std::isfinite(k_)) return (set_error("k must be positive and finite"), HH_EINVAL);
  if (n_ < 2 || n_ > 4096) return (set_error("n must be in [2, 4096]"), HH_EINVAL);
  if (strips < 1 || n_ % strips != 0) return (set_error("n must be a multiple of strips"), HH_EINVAL);
  if (n_ / strips < 2) return (set_error("each strip needs at least two node lines (n / strips >= 2)"), HH_EINVAL);
  if ((dirs & 15u) == 0 || (dirs & ~15u)) return (set_error("dirs must be a non-empty subset of HH_DIR_*"), HH_EINVAL);
  if (opts.precision != HH_PREC_FP32 && opts.precision != HH_PREC_FP64 && opts.precision != HH_PREC_BF16)
    return (set_error("bad precision"), HH_EINVAL);
  if (opts.precision == HH_PREC_BF16 && (!opts.tensor_cores || opts.interface_form != 1))
    return (set_error("HH_PREC_BF16 needs the tensor cores and interface_form 1"), HH_EINVAL);
  if (opts.maxit < 1 || opts.maxit > 2000) return (set_error("maxit must be in [1, 2000]"), HH_EINVAL);
  if (opts.bcr_depth < -1 || (opts.bcr_depth > 0 && (n_ % strips != 0 || opts.bcr_depth > max_bcr_depth(n_ / strips))))
    return (set_error("bcr_depth must be -1 (autotune), 0 (block Thomas) or d >= 1 with n / strips divisible by 2^d"),
            HH_EINVAL);
  if (opts.gs_passes != 1 && opts.gs_passes != 2) return (set_error("gs_passes must be 1 or 2"), HH_EINVAL);
  if (opts.gs_tensor != 0 && opts.gs_tensor != 1) return (set_error("gs_tensor must be 0 or 1"), HH_EINVAL);
  if (opts.twisted < -1 || opts.twisted > 1) return (set_error("twisted must be -1 (autotune), 0 or 1"), HH_EINVAL);
  if (opts.discretization != HH_DISC_P1 && opts.discretization != HH_DISC_FD)
    return (set_error("discretization must be HH_DISC_P1 or HH_DISC_FD"), HH_EINVAL);
  if (opts.discretization == HH_DISC_FD && opts.precision != HH_PREC_FP64)
    return (set_error("the five-point mode (HH_DISC_FD) runs in FP64 only"), HH_EINVAL);
  if (opts.serve_slots < 1 || opts.serve_slots > 256) return (set_error("serve_slots must be in 1..256"), HH_EINVAL);
  if (opts.interface_form != 0 && opts.interface_form != 1) return (set_error("interface_form must be 0 or 1"), HH_EINVAL);
  if (opts.timeout_cycles <= 0) opts.timeout_cycles = 4000000000LL;
  k = k_; n = n_; N = strips; m = n + 1; R = n / N;
  // bf16 sweeps: complex64 everywhere but in the products of the sweep (lowp.cu)
  lowp = opts.precision == HH_PREC_BF16;
  precision = lowp ? HH_PREC_FP32 : opts.precision;
  ldf = (m + 3) & ~3;
  coef.init(k, n);
  {
    // cyclic-reduction blocks: the requested depth, or every usable depth for the autotuner
    unsigned depths = 0;
    const int dl = max_bcr_depth(R);
    if (opts.bcr_depth > 0) depths = 1u << opts.bcr_depth;
    else if (opts.bcr_depth < 0)
      for (int d = 1; d <= dl; ++d) depths |= 1u << d;
    // the twisted strip solves run on the complex64 tensor-core kernels only, and a fixed
    // cyclic-reduction depth replaces them
    const bool twisted =
        opts.twisted != 0 && opts.bcr_depth <= 0 && precision == HH_PREC_FP32 && !lowp && opts.tensor_cores;
    bdir = block_directory(R, N, opts.interface_form, depths, twisted);
  }
  static const int bitcode[4] = {DC_LR, DC_RL, DC_BT, DC_TB};
  dir_codes.clear();
  for (int b = 0; b < 4; ++b)
    if (dirs & (1u << b)) dir_codes.push_back(bitcode[b]);
  t = (int)dir_codes.size();

  cudaError_t e = cudaGetDevice(&device);
  if (e != cudaSuccess) return (set_cuda_error(e, "cudaGetDevice"), HH_ECUDA);
  cudaDeviceProp prop;
  e = cudaGetDeviceProperties(&prop, device);
  if (e != cudaSuccess) return (set_cuda_error(e, "cudaGetDeviceProperties"), HH_ECUDA);
  num_sms = prop.multiProcessorCount;
  if (!prop.cooperativeLaunch) return (set_error("device does not support cooperative launches"), HH_ECUDA);
  if (opts.stream) {
    stream = (cudaStream_t)opts.stream;
  } else {
    e = cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return (set_cuda_error(e, "cudaStreamCreate"), HH_ECUDA);
    own_stream = true;
  }
  coop_per_sm = std::max(1, qr_blocks_per_sm());
  {
    // loads the module of the no-allocation entry point on this device, which reserves its
    // fixed scratch array now rather than at that entry point's first call
    void* scratch = nullptr;
    const int rc = noalloc_scratch_address(device, &scratch);
    if (rc) return rc;
  }

  if (opts.discretization == HH_DISC_FD) {
    // the paper's five-point scheme and overlapping strips: its own inverses and sweeps (fd.cu)
    if (dmalloc((void**)&bar, BAR_BYTES) || dmalloc((void**)&err, 64)) return HH_ENOMEM;
    cudaMemsetAsync(bar, 0, BAR_BYTES, stream);
    cudaMemsetAsync(err, 0, 64, stream);
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaEventRecord(a, stream);
    const int rc = fd_setup(*this);
    cudaEventRecord(b, stream);
    cudaEventSynchronize(b);
    float t_ms = 0;
    cudaEventElapsedTime(&t_ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    setup_ms_total = t_ms;
    collect_ticks();
    return rc;
  }
  const size_t fbytes = (size_t)factor_blocks() * m * ldf * sweep_elem();
  size_t free_b = 0, total_b = 0;
  cudaMemGetInfo(&free_b, &total_b);
  // the tensor-core form keeps two more copies of the complex64 factor store (hi and lo)
  const size_t fcopies = (precision == HH_PREC_FP32 && opts.tensor_cores) ? 3 : 1;
  if (fcopies * fbytes + (64ull << 20) > free_b)
    return (set_error("strip factors do not fit in free device memory"), HH_ENOMEM);
  if (dmalloc(&factors, fbytes) || dmalloc((void**)&bar, BAR_BYTES) || dmalloc((void**)&err, 64)) return HH_ENOMEM;
  cudaMemsetAsync(bar, 0, BAR_BYTES, stream);
  cudaMemsetAsync(err, 0, 64, stream);
  steps_double = build_steps(n, N, true);
  steps_single = build_steps(n, N, false);
  for (int d = 0; d <= bdir.dmax; ++d)
    if (d == 0 || bdir.iDeep[d] >= 0) {
      prog_double_d[d] = build_program(n, N, true, opts.interface_form, bdir, d);
      prog_single_d[d] = build_program(n, N, false, opts.interface_form, bdir, d);
    }
  if (bdir.iTw >= 0) {
    prog_double_d[PROG_TWISTED] = build_program(n, N, true, opts.interface_form, bdir, PROG_TWISTED);
    prog_single_d[PROG_TWISTED] = build_program(n, N, false, opts.interface_form, bdir, PROG_TWISTED);
  }
  if (upload_programs() || upload_persistent()) return HH_ENOMEM;
  cudaStreamSynchronize(stream);

  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  cudaEventRecord(a, stream);
  int rc = load_encoder();
  if (rc == HH_OK) rc = factor();
  if (rc == HH_OK) rc = prepare_tensor_cores();
  if (rc == HH_OK) rc = prepare_lowp();
  free_dense_scratch();
  cudaEventRecord(b, stream);
  cudaEventSynchronize(b);
  float t_ms = 0;
  cudaEventElapsedTime(&t_ms, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  setup_ms_total = t_ms;
  collect_ticks();
  return rc;
}

Engine::~Engine() {
  {
    std::lock_guard<std::mutex> lk(mu);
    stopping = true;
  }
  cv.notify_all();
  if (worker_started && worker.joinable()) worker.join();
  if (stream) cudaStreamSynchronize(stream);
  delete batch_solver;
  batch_solver = nullptr;
  for (auto& g : sweep_graphs) cudaGraphExecDestroy(g.exec);
  sweep_graphs.clear();
  collect_ticks();
  for (auto ev : event_pool) cudaEventDestroy(ev);
  fd_free(*this);
  dfree(factors); dfree(bar); dfree(err);
  dfree(w_rin); dfree(w_v); dfree(w_w); dfree(w_partial); dfree(w_t0); dfree(w_t1);
  dfree(prog_tasks);
  dfree(pprog_tasks);
  for (auto& kv : pphase_cache) dfree(kv.second);
  dfree(factors_hi); dfree(factors_lo); dfree(factors_bf16);
  dfree(stage_buf[0]); dfree(stage_buf[1]);
  free_dense_scratch();
  if (own_stream && stream) cudaStreamDestroy(stream);
}

// ------------------------------------------------------------------ host/device buffers
static bool is_device_ptr(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Stages a caller buffer on the device when it lives in host memory, in one of the handle's two
// staging buffers (slot 0 for an input, 1 for an output; grown on demand, kept for later calls,
// so that a call with host buffers allocates nothing once warm).  The handle's staging lock is
// held while the buffer is in use: calls on one handle from several threads take turns.
struct Staged {
  Engine* E;
  const void* user;
  void* dev = nullptr;
  size_t bytes;
  int slot;
  bool host;
  std::unique_lock<std::recursive_mutex> lk;
  Staged(Engine* e, const void* u, size_t b, int s) : E(e), user(u), bytes(b), slot(s) {
    host = !is_device_ptr(u);
    if (host) lk = std::unique_lock<std::recursive_mutex>(E->stage_mu);
  }
  int ensure() {
    if (E->stage_cap[slot] < bytes) {
      E->dfree(E->stage_buf[slot]);
      E->stage_buf[slot] = nullptr;
      E->stage_cap[slot] = 0;
      if (E->dmalloc(&E->stage_buf[slot], bytes)) return HH_ENOMEM;
      E->stage_cap[slot] = bytes;
    }
    dev = E->stage_buf[slot];
    return HH_OK;
  }
  int in() {
    if (!host) { dev = const_cast<void*>(user); return HH_OK; }
    if (ensure()) return HH_ENOMEM;
    cudaMemcpyAsync(dev, user, bytes, cudaMemcpyHostToDevice, E->stream);
    return HH_OK;
  }
  int alloc_out() {
    if (!host) { dev = const_cast<void*>(user); return HH_OK; }
    return ensure();
  }
  int out() {
    if (!host) return HH_OK;
    cudaMemcpyAsync(const_cast<void*>(user), dev, bytes, cudaMemcpyDeviceToHost, E->stream);
    cudaError_t e = cudaStreamSynchronize(E->stream);
    return e == cudaSuccess ? HH_OK : HH_ECUDA;
  }
  ~Staged() {
    if (host) cudaStreamSynchronize(E->stream);
  }
};

// ------------------------------------------------------------------ request loop
struct Engine::Request {
  const double* rhs;
  double* x;
  double tol;
  hh_result res;
  std::atomic<int> state{0};  // 0 queued, 1 running, 2 done
  hh_ticket id;
  std::chrono::steady_clock::time_point t_submit;
};

// The request loop: one thread per handle owning a SlotSolver of opts.serve_slots slots.
// Between two iterations it admits queued requests into the free slots; each iteration
// advances every active request by one MPGMRES step (one batched sweep launch over their
// columns); a request that finishes releases its slot at once.  solve_mu is held per
// iteration so blocking solves on the same handle interleave at iteration boundaries.
static void request_loop(Engine* Ep) {
  Engine& E = *Ep;
  cudaSetDevice(E.device);
  std::unique_ptr<SlotSolver> ss;
  std::vector<Engine::Request*> running;
  auto fail_all = [&](int rc) {
    for (auto* q : running) {
      std::memset(&q->res, 0, sizeof(q->res));
      q->res.status = (hh_status)rc;
      q->state = 2;
    }
    running.clear();
    ss.reset();
  };
  for (;;) {
    std::vector<Engine::Request*> take;
    {
      std::unique_lock<std::mutex> lk(E.mu);
      if (running.empty()) E.cv.wait(lk, [&] { return E.stopping || !E.queue.empty(); });
      if (E.stopping && running.empty()) return;
      if (!E.stopping) {
        const int room = E.opts.serve_slots - (int)running.size();
        while ((int)take.size() < room && !E.queue.empty()) {
          take.push_back(E.queue.front());
          E.queue.pop_front();
        }
      }
    }
    std::lock_guard<std::mutex> lk(E.solve_mu);
    if (!ss) {
      ss.reset(new SlotSolver(E));
      const int rc = ss->init(E.opts.serve_slots);
      if (rc) {
        for (auto* q : take) running.push_back(q);
        fail_all(rc);
        continue;
      }
    }
    if (!take.empty()) {
      const int nt = (int)take.size();
      std::vector<const double2*> b(nt);
      std::vector<double2*> x(nt);
      std::vector<double> tol(nt);
      std::vector<void*> tags(nt);
      for (int q = 0; q < nt; ++q) {
        b[q] = reinterpret_cast<const double2*>(take[q]->rhs);
        x[q] = reinterpret_cast<double2*>(take[q]->x);
        tol[q] = take[q]->tol;
        tags[q] = take[q];
        take[q]->state = 1;
        running.push_back(take[q]);
      }
      const int used = ss->admit(nt, b.data(), x.data(), tol.data(), tags.data(), nullptr);
      if (used < 0) {
        fail_all(-used);
        continue;
      }
    }
    std::vector<SlotDone> done;
    const int rc = ss->iterate(done);
    const auto now = std::chrono::steady_clock::now();
    for (auto& d : done) {
      auto* q = static_cast<Engine::Request*>(d.tag);
      q->res = d.res;
      q->res.t_setup_ms = E.setup_ms_total;
      q->res.t_solve_ms = std::chrono::duration<double, std::milli>(now - q->t_submit).count();
      running.erase(std::find(running.begin(), running.end(), q));
      q->state = 2;
    }
    if (rc) fail_all(rc);
  }
}

static std::mutex g_tickets_mu;
static std::unordered_map<hh_ticket, std::pair<Engine*, Engine::Request*>> g_tickets;
static std::atomic<uint64_t> g_next_ticket{1};

}  // namespace hh

using namespace hh;

struct hh_handle {
  Engine* E;
};

static int solve_common(hh_handle* h, int nrhs, const double* rhs, double* x, double tol, hh_result* res) {
  Engine& E = *h->E;
  if (!rhs || !x || nrhs < 1) return (set_error("rhs, x must be non-NULL and nrhs >= 1"), HH_EINVAL);
  if (!(tol > 0) || !std::isfinite(tol)) return (set_error("tol must be positive"), HH_EINVAL);
  std::lock_guard<std::mutex> lk(E.solve_mu);
  cudaSetDevice(E.device);
  const size_t bytes = (size_t)nrhs * E.m * E.m * sizeof(double2);
  auto t0 = std::chrono::steady_clock::now();
  Staged sb(&E, rhs, bytes, 0), sx(&E, x, bytes, 1);
  if (sb.in() || sx.alloc_out()) return HH_ENOMEM;
  std::vector<hh_result> tmp(nrhs);
  int rc = E.solve_batch_dev(nrhs, (const double2*)sb.dev, (double2*)sx.dev, tol, tmp.data());
  const bool have_x = rc == HH_OK || rc == HH_ENOCONV || rc == HH_EBREAKDOWN || rc == HH_ENAN;
  if (have_x && sx.out()) rc = HH_ECUDA;
  auto t1 = std::chrono::steady_clock::now();
  const double ms = std::chrono::duration<double, std::milli>(t1 - t0).count();
  for (int r = 0; r < nrhs; ++r) {
    tmp[r].t_setup_ms = E.setup_ms_total;
    tmp[r].t_solve_ms = ms;
    if (rc == HH_ECUDA || rc == HH_ENOMEM || rc == HH_ETIMEOUT) tmp[r].status = (hh_status)rc;
    if (res) res[r] = tmp[r];
  }
  return rc;
}

extern "C" {

void hh_default_opts(hh_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->precision = HH_PREC_FP64;
  o->scheme = HH_SCHEME_AUTO;
  o->single_sweep = 0;
  o->maxit = 200;
  o->deflate_eta = 1e-10;
  o->bcr_depth = 0;
  o->timeout_cycles = 4000000000LL;
  o->stream = nullptr;
  o->use_graph = 1;
  o->profile = 0;
  o->gs_passes = 2;
  o->serve_slots = 8;
  o->tensor_cores = 1;
  o->autotune = 1;
  o->fuse_chains = 1;
  o->overlap_steps = 1;
  o->interface_form = 1;
  o->persistent = 0;
  o->gs_first_fp32 = 1;
  o->gs_tensor = 1;
  o->group_wide_tiles = 1;
  o->twisted = 1;
}

hh_status hh_setup(double k, int n, int strips, uint32_t dirs, const hh_opts* opts, hh_handle** out) {
  if (!out) return (set_error("out must be non-NULL"), HH_EINVAL);
  *out = nullptr;
  Engine* E = new (std::nothrow) Engine();
  if (!E) return (set_error("out of host memory"), HH_ENOMEM);
  int rc = E->init(k, n, strips, dirs, opts);
  if (rc != HH_OK) {
    delete E;
    return (hh_status)rc;
  }
  *out = new hh_handle{E};
  return HH_OK;
}

hh_status hh_solve(hh_handle* h, const double* rhs, double* x, double tol, hh_result* res) {
  if (!h) return (set_error("NULL handle"), HH_EINVAL);
  return (hh_status)solve_common(h, 1, rhs, x, tol, res);
}

hh_status hh_solve_batch(hh_handle* h, int nrhs, const double* rhs, double* x, double tol, hh_result* res) {
  if (!h) return (set_error("NULL handle"), HH_EINVAL);
  return (hh_status)solve_common(h, nrhs, rhs, x, tol, res);
}

hh_status hh_assemble_rhs(hh_handle* h, int nsrc, const double* src, double* rhs) {
  if (!h || !rhs || (nsrc > 0 && !src) || nsrc < 0) return (set_error("bad arguments"), HH_EINVAL);
  Engine& E = *h->E;
  std::lock_guard<std::mutex> lk(E.solve_mu);
  cudaSetDevice(E.device);
  Staged so(&E, rhs, (size_t)E.m * E.m * sizeof(double2), 1);
  if (so.alloc_out()) return HH_ENOMEM;
  int rc = E.assemble_rhs(nsrc, src, (double2*)so.dev);
  if (rc == HH_OK && so.out()) rc = HH_ECUDA;
  return (hh_status)rc;
}

hh_status hh_apply_operator(hh_handle* h, int ncols, const double* x, double* y) {
  if (!h || !x || !y || ncols < 1) return (set_error("bad arguments"), HH_EINVAL);
  Engine& E = *h->E;
  std::lock_guard<std::mutex> lk(E.solve_mu);
  cudaSetDevice(E.device);
  const size_t bytes = (size_t)ncols * E.m * E.m * sizeof(double2);
  Staged sx(&E, x, bytes, 0), sy(&E, y, bytes, 1);
  if (sx.in() || sy.alloc_out()) return HH_ENOMEM;
  int rc = E.apply_operator(ncols, (const double2*)sx.dev, (double2*)sy.dev);
  if (rc == HH_OK && sy.out()) rc = HH_ECUDA;
  return (hh_status)rc;
}

hh_status hh_gram_schmidt_pass(hh_handle* h, int p, const double* V, int t, double* W, double* H) {
  if (!h || !V || !W || !H || p < 1 || t < 1 || t > 4) return (set_error("bad arguments"), HH_EINVAL);
  Engine& E = *h->E;
  std::lock_guard<std::mutex> lk(E.solve_mu);
  cudaSetDevice(E.device);
  const size_t col = (size_t)E.m * E.m * sizeof(double2);
  Staged sv(&E, V, (size_t)p * col, 0), sw(&E, W, (size_t)t * col, 1);
  if (sv.in() || sw.in()) return HH_ENOMEM;
  int rc = gram_schmidt_pass(E, p, (const double2*)sv.dev, t, (double2*)sw.dev, reinterpret_cast<double2*>(H));
  if (rc == HH_OK && sw.out()) rc = HH_ECUDA;
  return (hh_status)rc;
}

hh_status hh_apply_preconditioner(hh_handle* h, uint32_t dir, int ncols, const double* r, double* z) {
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
  std::lock_guard<std::mutex> lk(E.solve_mu);
  cudaSetDevice(E.device);
  const size_t bytes = (size_t)ncols * E.m * E.m * sizeof(double2);
  Staged sr(&E, r, bytes, 0), sz(&E, z, bytes, 1);
  if (sr.in() || sz.alloc_out()) return HH_ENOMEM;
  int rc = E.apply_preconditioner_dev(code, ncols, (const double2*)sr.dev, (double2*)sz.dev, E.opts.single_sweep != 0);
  if (rc == HH_OK && sz.out()) rc = HH_ECUDA;
  return (hh_status)rc;
}

hh_status hh_get_factor(hh_handle* h, int j, double* out) {
  if (!h || !out) return (set_error("bad arguments"), HH_EINVAL);
  Engine& E = *h->E;
  if (E.fd) return (set_error("the five-point mode keeps no P1 strip factors"), HH_EINVAL);
  if (j < 0 || j >= E.factor_blocks()) return (set_error("factor index out of range"), HH_EINVAL);
  std::lock_guard<std::mutex> lk(E.solve_mu);
  cudaSetDevice(E.device);
  const size_t cnt = (size_t)E.m * E.ldf;
  std::vector<double> full((size_t)E.m * E.m * 2);
  if (E.precision == HH_PREC_FP32) {
    std::vector<float2> tmp(cnt);
    cudaMemcpyAsync(tmp.data(), (const float2*)E.factors + (size_t)j * cnt, cnt * sizeof(float2), cudaMemcpyDeviceToHost, E.stream);
    if (cudaStreamSynchronize(E.stream) != cudaSuccess) return HH_ECUDA;
    for (int a = 0; a < E.m; ++a)
      for (int b = 0; b < E.m; ++b) {
        full[2 * ((size_t)a * E.m + b)] = tmp[(size_t)a * E.ldf + b].x;
        full[2 * ((size_t)a * E.m + b) + 1] = tmp[(size_t)a * E.ldf + b].y;
      }
  } else {
    std::vector<double2> tmp(cnt);
    cudaMemcpyAsync(tmp.data(), (const double2*)E.factors + (size_t)j * cnt, cnt * sizeof(double2), cudaMemcpyDeviceToHost, E.stream);
    if (cudaStreamSynchronize(E.stream) != cudaSuccess) return HH_ECUDA;
    for (int a = 0; a < E.m; ++a)
      for (int b = 0; b < E.m; ++b) {
        full[2 * ((size_t)a * E.m + b)] = tmp[(size_t)a * E.ldf + b].x;
        full[2 * ((size_t)a * E.m + b) + 1] = tmp[(size_t)a * E.ldf + b].y;
      }
  }
  const size_t bytes = full.size() * sizeof(double);
  if (is_device_ptr(out)) {
    cudaMemcpyAsync(out, full.data(), bytes, cudaMemcpyHostToDevice, E.stream);
    if (cudaStreamSynchronize(E.stream) != cudaSuccess) return HH_ECUDA;
  } else {
    std::memcpy(out, full.data(), bytes);
  }
  return HH_OK;
}

hh_status hh_get_stats(hh_handle* h, hh_stats* st) {
  if (!h || !st) return (set_error("bad arguments"), HH_EINVAL);
  Engine& E = *h->E;
  std::memset(st, 0, sizeof(*st));
  st->sweep_launches = E.launches[Engine::K_SWEEP];
  st->sweep_ms = E.ms[Engine::K_SWEEP];
  st->sweep_bytes = E.bytes[Engine::K_SWEEP];
  st->spmv_launches = E.launches[Engine::K_SPMV];
  st->spmv_ms = E.ms[Engine::K_SPMV];
  st->spmv_bytes = E.bytes[Engine::K_SPMV];
  st->gs_launches = E.launches[Engine::K_GS];
  st->gs_ms = E.ms[Engine::K_GS];
  st->gs_bytes = E.bytes[Engine::K_GS];
  st->setup_launches = E.launches[Engine::K_SETUP];
  st->setup_ms = E.setup_ms_total;
  st->setup_flops = E.flops[Engine::K_SETUP];
  st->kernel_launches = E.kernel_launches;
  st->factor_bytes = (int64_t)E.factor_blocks() * E.m * E.ldf * (int64_t)E.sweep_elem();
  st->factor_blocks = E.factor_blocks();
  if (E.fd) {  // the five-point mode: its chain of line-block inverses and the top ones
    st->factor_blocks = fd_blocks(E);
    st->factor_bytes = (int64_t)st->factor_blocks * E.m * E.ldf * (int64_t)sizeof(double2);
  }
  st->m = E.m;
  st->ldf = E.ldf;
  st->columns = E.last_columns;
  st->sweep_steps = (int64_t)E.program(E.last_columns, E.opts.single_sweep != 0).size();
  {
    const int d = E.depth_for(E.last_columns);
    st->bcr_depth = d == PROG_TWISTED ? 0 : d;
    st->twisted = d == PROG_TWISTED ? 1 : 0;
  }
  st->gemm_launches = E.launches[Engine::K_GEMM];
  st->gemm_ms = E.ms[Engine::K_GEMM];
  st->gemm_flops = E.flops[Engine::K_GEMM];
  st->tensor_cores = E.tc_ready ? 1 : 0;
  st->gsdot_launches = E.launches[Engine::K_GSDOT];
  st->gsdot_ms = E.ms[Engine::K_GSDOT];
  st->gsdot_flops = E.flops[Engine::K_GSDOT];
  st->gsdot_bytes = E.bytes[Engine::K_GSDOT];
  st->gs_flops = E.flops[Engine::K_GS];
  st->ns_blocks = E.ns_blocks;
  st->ns_iterations = E.ns_iterations;
  st->iterations_total = E.iterations_total;
  st->step_graphs = E.step_graphs_captured;
  st->step_graph_fallback = E.step_graph_fallback ? 1 : 0;
  {
    const auto it = E.tc_tuned.find(E.last_columns);
    if (it != E.tc_tuned.end()) {
      st->tc_bnc = it->second.shape == 1 ? 32 : (it->second.shape == 2 ? 128 : 64);
      st->tc_nsplit = it->second.nsplit;
      st->tc_cluster = it->second.cluster ? 1 : 0;
      st->tc_us = it->second.us;
    }
  }
  for (const SweepPhase& ph : E.program(E.last_columns, E.opts.single_sweep != 0))
    st->wide_steps += (int64_t)(ph.kind == PH_GROUP || (ph.kind == PH_STEP && ph.step.ns * E.last_columns > 8));
  return HH_OK;
}

void hh_reset_stats(hh_handle* h) {
  if (!h) return;
  Engine& E = *h->E;
  for (int c = 0; c < Engine::K_NCLASS; ++c) {
    if (c == Engine::K_SETUP) continue;
    E.launches[c] = 0; E.ms[c] = 0; E.bytes[c] = 0; E.flops[c] = 0;
  }
  E.kernel_launches = 0;
  E.iterations_total = 0;
}

hh_status hh_submit(hh_handle* h, const double* rhs, double* x, double tol, hh_ticket* ticket) {
  if (!h || !rhs || !x || !ticket) return (set_error("bad arguments"), HH_EINVAL);
  if (!(tol > 0)) return (set_error("tol must be positive"), HH_EINVAL);
  Engine& E = *h->E;
  auto* rq = new Engine::Request();
  rq->rhs = rhs; rq->x = x; rq->tol = tol;
  rq->id = g_next_ticket++;
  rq->t_submit = std::chrono::steady_clock::now();
  std::memset(&rq->res, 0, sizeof(rq->res));
  {
    std::lock_guard<std::mutex> lk(g_tickets_mu);
    g_tickets[rq->id] = {&E, rq};
  }
  {
    std::lock_guard<std::mutex> lk(E.mu);
    E.queue.push_back(rq);
    if (!E.worker_started) {
      E.worker_started = true;
      E.worker = std::thread(request_loop, &E);
    }
  }
  E.cv.notify_all();
  *ticket = rq->id;
  return HH_OK;
}

hh_status hh_poll(hh_ticket ticket, hh_result* res) {
  Engine::Request* rq = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_tickets_mu);
    auto it = g_tickets.find(ticket);
    if (it == g_tickets.end()) return (set_error("unknown ticket"), HH_EINVAL);
    rq = it->second.second;
    if (rq->state.load() != 2) return HH_EPENDING;
    g_tickets.erase(it);
  }
  if (res) *res = rq->res;
  hh_status st = rq->res.status;
  delete rq;
  return st;
}

void hh_destroy(hh_handle* h) {
  if (!h) return;
  {
    std::lock_guard<std::mutex> lk(g_tickets_mu);
    for (auto it = g_tickets.begin(); it != g_tickets.end();) {
      if (it->second.first == h->E && it->second.second->state.load() == 0) {
        std::lock_guard<std::mutex> lk2(h->E->mu);
        for (auto q = h->E->queue.begin(); q != h->E->queue.end(); ++q)
          if (*q == it->second.second) { h->E->queue.erase(q); break; }
        delete it->second.second;
        it = g_tickets.erase(it);
      } else {
        ++it;
      }
    }
  }
  delete h->E;
  delete h;
}

const char* hh_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
