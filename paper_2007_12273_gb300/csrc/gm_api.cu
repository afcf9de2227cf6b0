// gm_api.cu -- the C ABI (include/gm.h): argument checks, the internal
// workspace, launch configuration and error reporting.
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "gm_kernels.cuh"
#include "std_kernel.cuh"

namespace gmcr {
int em_blocks_per_sm_d1(int nt, int fp64_mstep, int v_f64, size_t smem);
int em_blocks_per_sm_d3(int nt, int fp64_mstep, int v_f64, size_t smem);
}  // namespace gmcr

namespace {

thread_local std::string g_err;

// a capture in progress on this host thread (gm_graph_begin .. gm_graph_end):
// workspace requests get buffers of their own, handed to the graph
struct Capture {
  bool active = false;
  cudaStream_t stream = nullptr;
  std::vector<void*> bufs;
};
thread_local Capture g_cap;

std::mutex g_ws_mu;
void* g_ws = nullptr;
size_t g_ws_bytes = 0;
int g_ws_dev = -1;

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  return fail(GM_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

// the kernels are built for sm_103a only
int check_device(int* sm_count) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  int major = 0, minor = 0, sms = 0;
  if ((e = cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev)) != cudaSuccess ||
      (e = cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev)) != cudaSuccess ||
      (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
    return cuda_fail(e, "cudaDeviceGetAttribute");
  if (major != 10 || minor != 3)
    return fail(GM_ERR_UNSUPPORTED, "device %d has compute capability %d.%d; this library is built for sm_103a",
                dev, major, minor);
  if (sm_count) *sm_count = sms;
  return GM_OK;
}

// grows the single workspace; the old buffer is released with cudaFree,
// which waits for work that may still use it
int ws_get(size_t bytes, void** out) {
  if (g_cap.active) {  // owned by the graph being captured
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, bytes > 0 ? bytes : 256);
    if (e != cudaSuccess) return fail(GM_ERR_NOMEM, "graph workspace of %zu bytes: %s", bytes,
                                      cudaGetErrorString(e));
    g_cap.bufs.push_back(p);
    *out = p;
    return GM_OK;
  }
  std::lock_guard<std::mutex> lk(g_ws_mu);
  int dev = 0;
  cudaGetDevice(&dev);
  if (g_ws && (bytes > g_ws_bytes || dev != g_ws_dev)) {
    int cur = dev;
    cudaSetDevice(g_ws_dev);
    cudaFree(g_ws);
    cudaSetDevice(cur);
    g_ws = nullptr;
    g_ws_bytes = 0;
  }
  if (!g_ws) {
    const size_t want = bytes + bytes / 4 + 4096;
    cudaError_t e = cudaMalloc(&g_ws, want);
    if (e != cudaSuccess) {
      g_ws = nullptr;
      return fail(GM_ERR_NOMEM, "workspace of %zu bytes: %s", want, cudaGetErrorString(e));
    }
    g_ws_bytes = want;
    g_ws_dev = dev;
  }
  *out = g_ws;
  return GM_OK;
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

int check_cfg(const gm_config* cfg) {
  if (!cfg) return fail(GM_ERR_ARG, "cfg is NULL");
  if (cfg->D != 1 && cfg->D != 3) return fail(GM_ERR_ARG, "D must be 1 or 3 (got %d)", cfg->D);
  if (cfg->Kmax < 1 || cfg->Kmax > gmcr::kMaxK)
    return fail(GM_ERR_ARG, "Kmax must be in 1..%d (got %d)", gmcr::kMaxK, cfg->Kmax);
  if (cfg->shape_order != 1 && cfg->shape_order != 2)
    return fail(GM_ERR_ARG, "shape_order must be 1 or 2 (got %d)", cfg->shape_order);
  if (!(cfg->L > 0.0)) return fail(GM_ERR_ARG, "L must be positive");
  return GM_OK;
}

// the argument checks of gm_reconstruct (and of gm_reconstruct_noalloc),
// up to the device check; nothing is launched
int check_reconstruct(const gm_config* cfg, int64_t C, const int32_t* K, const double* params,
                      const double* W, const double* rho_target, int64_t n_out,
                      const int64_t* out_off, const double* x_out, const double* v_out,
                      const double* alpha_out, const uint32_t* status_out) {
  int rc = check_cfg(cfg);
  if (rc) return rc;
  if (!(cfg->q != 0.0)) return fail(GM_ERR_ARG, "q must be nonzero (the mass matrix is q times the shape sums)");
  if (C < 0) return fail(GM_ERR_ARG, "C < 0");
  if (n_out < 0 || n_out >= (int64_t)1 << 40) return fail(GM_ERR_ARG, "n_out out of range");
  if (C == 0) return GM_OK;
  if (!K || !params || !W || !rho_target || !out_off || !status_out)
    return fail(GM_ERR_ARG, "a required pointer is NULL");
  if (n_out > 0 && (!x_out || !v_out || !alpha_out))
    return fail(GM_ERR_ARG, "an output particle pointer is NULL");
  return GM_OK;
}

}  // namespace

int gmcr::api_check_reconstruct(const gm_config* cfg, int64_t C, const int32_t* K,
                                const double* params, const double* W, const double* rho_target,
                                int64_t n_out, const int64_t* out_off, const double* x_out,
                                const double* v_out, const double* alpha_out,
                                const uint32_t* status_out) {
  return check_reconstruct(cfg, C, K, params, W, rho_target, n_out, out_off, x_out, v_out,
                           alpha_out, status_out);
}

int gmcr::api_check_device() { return check_device(nullptr); }

int gmcr::record_error(int code, const char* msg) {
  g_err = msg;
  return code;
}

struct gm_graph {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<void*> bufs;
};

extern "C" {

const char* gm_last_error(void) { return g_err.c_str(); }

int gm_graph_begin(void* stream) {
  g_err.clear();
  if (g_cap.active) return fail(GM_ERR_ARG, "a capture is already in progress on this thread");
  int rc = check_device(nullptr);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamBeginCapture");
  g_cap.active = true;
  g_cap.stream = s;
  g_cap.bufs.clear();
  return GM_OK;
}

int gm_graph_end(void* stream, gm_graph** out) {
  g_err.clear();
  if (!g_cap.active) return fail(GM_ERR_ARG, "no capture in progress on this thread");
  cudaStream_t s = (cudaStream_t)stream;
  if (s != g_cap.stream) return fail(GM_ERR_ARG, "gm_graph_end on another stream than gm_graph_begin");
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(s, &graph);
  g_cap.active = false;
  std::vector<void*> bufs;
  bufs.swap(g_cap.bufs);
  auto release = [&]() {
    if (graph) cudaGraphDestroy(graph);
    for (void* p : bufs) cudaFree(p);
  };
  if (e != cudaSuccess) {
    release();
    return cuda_fail(e, "cudaStreamEndCapture");
  }
  if (!out) {
    release();
    return fail(GM_ERR_ARG, "out is NULL");
  }
  cudaGraphExec_t exec = nullptr;
  e = cudaGraphInstantiate(&exec, graph, 0);
  if (e != cudaSuccess) {
    release();
    return cuda_fail(e, "cudaGraphInstantiate");
  }
  gm_graph* g = new gm_graph;
  g->graph = graph;
  g->exec = exec;
  g->bufs.swap(bufs);
  *out = g;
  return GM_OK;
}

int gm_graph_launch(const gm_graph* g, void* stream) {
  g_err.clear();
  if (!g) return fail(GM_ERR_ARG, "graph is NULL");
  cudaError_t e = cudaGraphLaunch(g->exec, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
  return GM_OK;
}

int gm_graph_destroy(gm_graph* g) {
  g_err.clear();
  if (!g) return GM_OK;
  cudaDeviceSynchronize();
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  for (void* p : g->bufs) cudaFree(p);
  delete g;
  return GM_OK;
}

int gm_shutdown(void) {
  std::lock_guard<std::mutex> lk(g_ws_mu);
  if (g_ws) {
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(g_ws_dev);
    cudaFree(g_ws);
    cudaSetDevice(cur);
  }
  g_ws = nullptr;
  g_ws_bytes = 0;
  g_ws_dev = -1;
  return GM_OK;
}

static int compress_impl(const gm_config* cfg, int64_t C, int64_t n_particles,
                         const int64_t* cell_off, const double* x, const void* v, int32_t v_is_f64,
                         const double* alpha, const int32_t* init_K, const double* init_params,
                         int32_t* K_out, double* params_out, double* W_out,
                         double* rho_target_out, double* lnL_out, int32_t* sweeps_out,
                         int32_t* kwork_out, uint32_t* status_out, void* stream) {
  g_err.clear();
  int rc = check_cfg(cfg);
  if (rc) return rc;
  if (C < 0 || C >= (int64_t)1 << 31) return fail(GM_ERR_ARG, "C out of range (%lld)", (long long)C);
  if (n_particles < 0) return fail(GM_ERR_ARG, "n_particles < 0");
  if (cfg->max_sweeps < 1) return fail(GM_ERR_ARG, "max_sweeps must be >= 1");
  if (!(cfg->tol >= 0.0)) return fail(GM_ERR_ARG, "tol must be >= 0");
  if (C == 0) return GM_OK;
  if (!cell_off || !v || !alpha || !K_out || !params_out || !W_out || !lnL_out || !status_out)
    return fail(GM_ERR_ARG, "a required pointer is NULL");
  if (!x != !rho_target_out) return fail(GM_ERR_ARG, "x and rho_target_out must be both set or both NULL");
  const int D = cfg->D;
  int nt = cfg->threads_per_cell > 0 ? cfg->threads_per_cell : 256;
  if (nt != 64 && nt != 128 && nt != 256)
    return fail(GM_ERR_ARG, "threads_per_cell must be 64, 128 or 256");
  int cap = cfg->smem_particles > 0 ? cfg->smem_particles : (D == 1 ? 2560 : 3072);
  cap &= ~3;  // pair records of 16 bytes behind D arrays of cap floats
  if (cap < 4) cap = 4;
  const size_t smem = (size_t)cap * (D + 4) * sizeof(float);
  if (smem > 200 * 1024) return fail(GM_ERR_ARG, "smem_particles too large (%d)", cap);
  if (cfg->precision != 0 && cfg->precision != 1)
    return fail(GM_ERR_ARG, "precision must be 0 (FP64 M-step) or 1 (FP32) (got %d)", cfg->precision);
  const int fp64_mstep = cfg->precision == 0;
  int sms = 0;
  if ((rc = check_device(&sms))) return rc;
  cudaStream_t s = (cudaStream_t)stream;

  const size_t q_bytes = 256, part_bytes = align256(gmcr::deposit_ws_bytes(C));
  const size_t list_bytes = init_K ? align256((size_t)C * sizeof(unsigned int)) : 0;
  const int64_t sstride = gmcr::scratch_stride(n_particles, C);
  if ((int64_t)(D + 4) * sstride >= ((int64_t)1 << 31))
    return fail(GM_ERR_ARG, "too many particles for one call (%lld)", (long long)n_particles);
  const size_t scr_bytes = align256((size_t)sstride * (D + 4) * sizeof(float));
  const size_t k1_bytes = init_K ? align256(gmcr::em_k1_raw_bytes(D, C)) : 0;
  void* ws = nullptr;
  if ((rc = ws_get(q_bytes + part_bytes + list_bytes + scr_bytes + k1_bytes, &ws))) return rc;
  char* wb = (char*)ws;
  unsigned int* queue = (unsigned int*)wb;
  unsigned int* list_count = queue + 1;
  double* part = (double*)(wb + q_bytes);
  unsigned int* list = init_K ? (unsigned int*)(wb + q_bytes + part_bytes) : nullptr;
  float* scratch = (float*)(wb + q_bytes + part_bytes + list_bytes);
  void* k1_raw = init_K ? (void*)(wb + q_bytes + part_bytes + list_bytes + scr_bytes) : nullptr;

  cudaError_t e = cudaMemsetAsync(queue, 0, 2 * sizeof(unsigned int), s);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
  gmcr::trace_mark(nullptr, s);
  gmcr::EmParams p;
  p.C = C;
  p.n = n_particles;
  p.cell_off = cell_off;
  p.v = v;
  p.alpha = alpha;
  p.K_out = K_out;
  p.params_out = params_out;
  p.W_out = W_out;
  p.lnL_out = lnL_out;
  p.sweeps_out = sweeps_out;
  p.kwork_out = kwork_out;
  p.status_out = status_out;
  p.init_K = init_K;
  p.init_prm = init_params;
  p.scratch = scratch;
  p.scratch_stride = sstride;
  p.queue = queue;
  p.list = list;
  p.list_count = list_count;
  p.Kmax = cfg->Kmax;
  p.max_sweeps = cfg->max_sweeps;
  p.cap = cap;
  p.tol = cfg->tol;
  p.seed = cfg->seed;
  const int per_sm = D == 1 ? gmcr::em_blocks_per_sm_d1(nt, fp64_mstep, v_is_f64, smem)
                            : gmcr::em_blocks_per_sm_d3(nt, fp64_mstep, v_is_f64, smem);
  if (per_sm < 1) return fail(GM_ERR_CUDA, "EM kernel does not fit on an SM (smem %zu)", smem);
  int64_t grid = (int64_t)per_sm * sms;
  if (grid > C) grid = C;
  if (init_K) {
    // supplied starts: the closed-form cells (one valid component, empty,
    // degenerate) one warp each; the EM kernel takes the list of the rest
    gmcr::K1Params kp;
    kp.C = C;
    kp.n = n_particles;
    kp.cell_off = cell_off;
    kp.v = v;
    kp.alpha = alpha;
    kp.init_K = init_K;
    kp.init_prm = init_params;
    kp.K_out = K_out;
    kp.params_out = params_out;
    kp.W_out = W_out;
    kp.lnL_out = lnL_out;
    kp.sweeps_out = sweeps_out;
    kp.kwork_out = kwork_out;
    kp.status_out = status_out;
    kp.list = list;
    kp.list_count = list_count;
    kp.raw = k1_raw;
    // the charge deposit rides along (one read of the weights)
    kp.x = x;
    kp.inv_dx = 1.0 / (cfg->L / (double)C);
    kp.order = cfg->shape_order;
    kp.dep_rec = x ? (long long*)part : nullptr;
    kp.Kmax = cfg->Kmax;
    e = gmcr::launch_em_k1(D, v_is_f64, kp, sms, s);
    if (e != cudaSuccess) return cuda_fail(e, "closed-form pre-pass launch");
  }
  e = D == 1 ? gmcr::launch_em1(p, nt, fp64_mstep, v_is_f64, smem, (int)grid, s)
             : gmcr::launch_em3(p, nt, fp64_mstep, v_is_f64, smem, (int)grid, s);
  if (e != cudaSuccess) return cuda_fail(e, "EM kernel launch");
  gmcr::trace_mark("em_kernel", s);
  if (x && init_K) {  // the records came from em_k1_kernel
    e = gmcr::launch_deposit_combine(C, cfg->L / (double)C, cfg->q, cfg->shape_order, part,
                                     rho_target_out, s);
    if (e != cudaSuccess) return cuda_fail(e, "deposit launch");
    gmcr::trace_mark("deposit_combine_kernel", s);
  } else if (x) {
    e = gmcr::launch_deposit(C, cell_off, x, alpha, cfg->L / (double)C, cfg->q, cfg->shape_order,
                             part, rho_target_out, s);
    if (e != cudaSuccess) return cuda_fail(e, "deposit launch");
    gmcr::trace_mark("deposit (deposit_partials_kernel, deposit_combine_kernel)", s);
  }
  return GM_OK;
}

int gm_compress(const gm_config* cfg, int64_t C, int64_t n_particles, const int64_t* cell_off,
                const double* x, const void* v, int32_t v_is_f64, const double* alpha,
                int32_t* K_out, double* params_out, double* W_out, double* rho_target_out,
                double* lnL_out, int32_t* sweeps_out, int32_t* kwork_out, uint32_t* status_out,
                void* stream) {
  return compress_impl(cfg, C, n_particles, cell_off, x, v, v_is_f64, alpha, nullptr, nullptr,
                       K_out, params_out, W_out, rho_target_out, lnL_out, sweeps_out, kwork_out,
                       status_out, stream);
}

int gm_compress_standard(const gm_config* cfg, const gm_std_opts* opts, int64_t C,
                         int64_t n_particles, const int64_t* cell_off, const double* x,
                         const void* v, int32_t v_is_f64, const double* alpha, int32_t* K_out,
                         double* params_out, double* W_out, double* rho_target_out,
                         double* lnL_out, int32_t* iters_out, int32_t* aa_steps_out,
                         int32_t* aa_resets_out, int32_t* km_passes_out, uint32_t* status_out,
                         void* stream) {
  g_err.clear();
  int rc = check_cfg(cfg);
  if (rc) return rc;
  if (!opts) return fail(GM_ERR_ARG, "opts is NULL");
  if (opts->init != 0 && opts->init != 1) return fail(GM_ERR_ARG, "opts->init must be 0 or 1");
  if (opts->aa_memory < 0 || opts->aa_memory > gmcr::kStdMaxM)
    return fail(GM_ERR_ARG, "opts->aa_memory must be in 0..%d", gmcr::kStdMaxM);
  if (opts->kmeans_iters < 0) return fail(GM_ERR_ARG, "opts->kmeans_iters < 0");
  if (opts->penalised != 0 && opts->penalised != 1) return fail(GM_ERR_ARG, "opts->penalised must be 0 or 1");
  if (opts->penalised && opts->aa_memory)
    return fail(GM_ERR_ARG, "opts->aa_memory must be 0 with opts->penalised");
  if (C < 0 || C >= (int64_t)1 << 31) return fail(GM_ERR_ARG, "C out of range (%lld)", (long long)C);
  if (n_particles < 0) return fail(GM_ERR_ARG, "n_particles < 0");
  if (cfg->max_sweeps < 1) return fail(GM_ERR_ARG, "max_sweeps must be >= 1");
  if (!(cfg->tol >= 0.0)) return fail(GM_ERR_ARG, "tol must be >= 0");
  if (C == 0) return GM_OK;
  if (!cell_off || !v || !alpha || !K_out || !params_out || !W_out || !lnL_out || !status_out)
    return fail(GM_ERR_ARG, "a required pointer is NULL");
  if (!x != !rho_target_out) return fail(GM_ERR_ARG, "x and rho_target_out must be both set or both NULL");
  int sms = 0;
  if ((rc = check_device(&sms))) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  const int D = cfg->D;
  int cap = cfg->smem_particles > 0 ? cfg->smem_particles : (D == 1 ? 2560 : 3072);
  cap &= ~3;
  if (cap < 4) cap = 4;
  const size_t smem = (size_t)cap * (D + 3) * sizeof(float);
  if (smem > 160 * 1024) return fail(GM_ERR_ARG, "smem_particles too large (%d)", cap);

  const size_t q_bytes = 256, part_bytes = align256(gmcr::deposit_ws_bytes(C));
  const int64_t sstride = gmcr::scratch_stride(n_particles, C);
  if ((int64_t)(D + 3) * sstride >= ((int64_t)1 << 31))
    return fail(GM_ERR_ARG, "too many particles for one call (%lld)", (long long)n_particles);
  const size_t scr_bytes = align256((size_t)sstride * (D + 3) * sizeof(float));
  void* ws = nullptr;
  if ((rc = ws_get(q_bytes + part_bytes + scr_bytes, &ws))) return rc;
  char* wb = (char*)ws;
  unsigned int* queue = (unsigned int*)wb;
  double* part = (double*)(wb + q_bytes);
  float* scratch = (float*)(wb + q_bytes + part_bytes);
  cudaError_t e = cudaMemsetAsync(queue, 0, sizeof(unsigned int), s);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
  gmcr::StdParams p;
  p.C = C;
  p.n = n_particles;
  p.cell_off = cell_off;
  p.v = v;
  p.alpha = alpha;
  p.K_out = K_out;
  p.params_out = params_out;
  p.W_out = W_out;
  p.lnL_out = lnL_out;
  p.iters_out = iters_out;
  p.aa_steps_out = aa_steps_out;
  p.aa_resets_out = aa_resets_out;
  p.km_out = km_passes_out;
  p.status_out = status_out;
  p.scratch = scratch;
  p.scratch_stride = sstride;
  p.queue = queue;
  p.Kmax = cfg->Kmax;
  p.max_sweeps = cfg->max_sweeps;
  p.cap = cap;
  p.init = opts->init;
  p.aa_m = opts->aa_memory;
  p.km_iters = opts->kmeans_iters;
  p.mml = opts->penalised;
  p.tol = cfg->tol;
  p.seed = cfg->seed;
  e = gmcr::launch_std(D, p, v_is_f64, smem, sms, s);
  if (e != cudaSuccess) return cuda_fail(e, "standard EM kernel launch");
  if (x) {
    e = gmcr::launch_deposit(C, cell_off, x, alpha, cfg->L / (double)C, cfg->q, cfg->shape_order,
                             part, rho_target_out, s);
    if (e != cudaSuccess) return cuda_fail(e, "deposit launch");
  }
  return GM_OK;
}

int gm_anderson_affine(int32_t n, const double* A, const double* b, const double* x0,
                       int32_t memory, int32_t iters, double* x_out, double* res_out,
                       void* stream) {
  g_err.clear();
  if (n < 1 || n > gmcr::kMaxK * 10) return fail(GM_ERR_ARG, "n must be in 1..%d", gmcr::kMaxK * 10);
  if (memory < 0 || memory > gmcr::kStdMaxM) return fail(GM_ERR_ARG, "memory must be in 0..%d", gmcr::kStdMaxM);
  if (iters < 0) return fail(GM_ERR_ARG, "iters < 0");
  if (!A || !b || !x0 || !x_out || (iters > 0 && !res_out)) return fail(GM_ERR_ARG, "a required pointer is NULL");
  int rc = check_device(nullptr);
  if (rc) return rc;
  cudaError_t e = gmcr::launch_aa_affine(n, A, b, x0, memory, iters, x_out, res_out, (cudaStream_t)stream);
  return e == cudaSuccess ? GM_OK : cuda_fail(e, "Anderson kernel launch");
}

int gm_compress_from(const gm_config* cfg, int64_t C, int64_t n_particles,
                     const int64_t* cell_off, const double* x, const void* v, int32_t v_is_f64,
                     const double* alpha, const int32_t* init_K, const double* init_params,
                     int32_t* K_out, double* params_out, double* W_out, double* rho_target_out,
                     double* lnL_out, int32_t* sweeps_out, int32_t* kwork_out,
                     uint32_t* status_out, void* stream) {
  if (!init_K || !init_params) return fail(GM_ERR_ARG, "init_K and init_params are required");
  return compress_impl(cfg, C, n_particles, cell_off, x, v, v_is_f64, alpha, init_K, init_params,
                       K_out, params_out, W_out, rho_target_out, lnL_out, sweeps_out, kwork_out,
                       status_out, stream);
}

int gm_reconstruct(const gm_config* cfg, int64_t C, const int32_t* K, const double* params,
                   const double* W, const double* rho_target, int64_t n_out,
                   const int64_t* out_off, double* x_out, double* v_out, double* alpha_out,
                   uint32_t* status_out, double* dA_out, void* stream) {
  g_err.clear();
  int rc = check_reconstruct(cfg, C, K, params, W, rho_target, n_out, out_off, x_out, v_out,
                             alpha_out, status_out);
  if (rc) return rc;
  if (C == 0) return GM_OK;
  if ((rc = check_device(nullptr))) return rc;
  void* ws = nullptr;
  if ((rc = ws_get(gmcr::reconstruct_ws_bytes(cfg->D, C, cfg->Kmax), &ws))) return rc;
  cudaError_t e = gmcr::launch_reconstruct(cfg->D, C, cfg->Kmax, K, params, W, rho_target, n_out,
                                           out_off, cfg->seed, cfg->L / (double)C, cfg->q,
                                           cfg->shape_order, x_out, v_out, alpha_out, status_out,
                                           dA_out, ws, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "reconstruct launch");
  return GM_OK;
}

static int check_mesh2d(const gm_mesh2d* mesh) {
  if (!mesh) return fail(GM_ERR_ARG, "mesh is NULL");
  if (mesh->Cx < 1 || mesh->Cy < 1 || mesh->Cx > ((int64_t)1 << 24) || mesh->Cy > ((int64_t)1 << 24) ||
      mesh->Cx * mesh->Cy >= ((int64_t)1 << 31))
    return fail(GM_ERR_ARG, "mesh size out of range (%lld x %lld)", (long long)mesh->Cx,
                (long long)mesh->Cy);
  if (!(mesh->Lx > 0.0) || !(mesh->Ly > 0.0)) return fail(GM_ERR_ARG, "Lx and Ly must be positive");
  return GM_OK;
}

int gm_deposit_2d(const gm_config* cfg, const gm_mesh2d* mesh, const int64_t* cell_off,
                  const double* x, const double* y, const double* alpha, double* rho_out,
                  void* stream) {
  g_err.clear();
  int rc = check_cfg(cfg);
  if (rc) return rc;
  if ((rc = check_mesh2d(mesh))) return rc;
  if (!cell_off || !x || !y || !rho_out) return fail(GM_ERR_ARG, "a required pointer is NULL");
  if ((rc = check_device(nullptr))) return rc;
  const int64_t C = mesh->Cx * mesh->Cy;
  void* ws = nullptr;
  if ((rc = ws_get(align256((size_t)9 * C * sizeof(double)), &ws))) return rc;
  cudaError_t e = gmcr::launch_deposit2d(mesh->Cx, mesh->Cy, cell_off, x, y, alpha,
                                         mesh->Lx / (double)mesh->Cx, mesh->Ly / (double)mesh->Cy,
                                         cfg->q, cfg->shape_order, (double*)ws, rho_out,
                                         (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "2D deposit launch");
  return GM_OK;
}

int gm_reconstruct_2d(const gm_config* cfg, const gm_mesh2d* mesh, const int32_t* K,
                      const double* params, const double* W, const double* rho_target,
                      int64_t n_out, const int64_t* out_off, double* x_out, double* y_out,
                      double* v_out, double* alpha_out, uint32_t* status_out, double* dA_out,
                      void* stream) {
  g_err.clear();
  int rc = check_cfg(cfg);
  if (rc) return rc;
  if ((rc = check_mesh2d(mesh))) return rc;
  if (!(cfg->q != 0.0)) return fail(GM_ERR_ARG, "q must be nonzero");
  if (n_out < 0 || n_out >= (int64_t)1 << 40) return fail(GM_ERR_ARG, "n_out out of range");
  if (!K || !params || !W || !rho_target || !out_off || !status_out)
    return fail(GM_ERR_ARG, "a required pointer is NULL");
  if (n_out > 0 && (!x_out || !y_out || !v_out || !alpha_out))
    return fail(GM_ERR_ARG, "an output particle pointer is NULL");
  if ((rc = check_device(nullptr))) return rc;
  void* ws = nullptr;
  if ((rc = ws_get(gmcr::reconstruct2d_ws_bytes(cfg->D, mesh->Cx, mesh->Cy), &ws))) return rc;
  cudaError_t e = gmcr::launch_reconstruct2d(
      cfg->D, mesh->Cx, mesh->Cy, cfg->Kmax, K, params, W, rho_target, n_out, out_off, cfg->seed,
      mesh->Lx / (double)mesh->Cx, mesh->Ly / (double)mesh->Cy, cfg->q, cfg->shape_order, x_out,
      y_out, v_out, alpha_out, status_out, dA_out, ws, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "2D reconstruct launch");
  return GM_OK;
}

int gm_moments(const gm_config* cfg, int64_t C, int64_t n_particles, const int64_t* cell_off,
               const double* x, const void* v, int32_t v_is_f64, const double* alpha, double* W,
               double* p, double* M2, double* E, double* rho, void* stream) {
  g_err.clear();
  int rc = check_cfg(cfg);
  if (rc) return rc;
  if (C < 0 || n_particles < 0) return fail(GM_ERR_ARG, "negative size");
  if (C == 0) return GM_OK;
  if (!cell_off || !alpha || (!v && (p || M2 || E)) || (!x && rho))
    return fail(GM_ERR_ARG, "a required pointer is NULL");
  if ((rc = check_device(nullptr))) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaSuccess;
  if (W || p || M2 || E) {
    e = gmcr::launch_moments(cfg->D, C, n_particles, cell_off, v, v_is_f64, alpha, W, p, M2, E, s);
    if (e != cudaSuccess) return cuda_fail(e, "moments launch");
  }
  if (rho) {
    void* ws = nullptr;
    if ((rc = ws_get(align256(gmcr::deposit_ws_bytes(C)), &ws))) return rc;
    e = gmcr::launch_deposit(C, cell_off, x, alpha, cfg->L / (double)C, cfg->q, cfg->shape_order,
                             ws, rho, s);
    if (e != cudaSuccess) return cuda_fail(e, "deposit launch");
  }
  return GM_OK;
}

int gm_mixture_moments(const gm_config* cfg, int64_t C, const int32_t* K, const double* params,
                       const double* Wc, double* W, double* p, double* M2, double* E,
                       void* stream) {
  g_err.clear();
  int rc = check_cfg(cfg);
  if (rc) return rc;
  if (C < 0) return fail(GM_ERR_ARG, "C < 0");
  if (C == 0) return GM_OK;
  if (!K || !params || !Wc) return fail(GM_ERR_ARG, "a required pointer is NULL");
  if ((rc = check_device(nullptr))) return rc;
  cudaError_t e = gmcr::launch_mixture_moments(cfg->D, C, cfg->Kmax, K, params, Wc, W, p, M2, E,
                                               (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "mixture moments launch");
  return GM_OK;
}

}  // extern "C"
