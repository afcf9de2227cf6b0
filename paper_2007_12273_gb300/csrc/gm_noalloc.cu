// gm_noalloc.cu -- gm_reconstruct_noalloc: the reconstruction of
// gm_reconstruct with its scratch in a fixed, statically allocated device
// array instead of the library's growable workspace.
//
// For callers that cannot allocate device memory while they run: a host
// code whose device memory is owned by its own allocator or by a fixed
// budget, or one that must not pay the device-wide synchronisation of
// cudaFree/cudaMalloc (gm_reconstruct grows its workspace that way).  The
// library itself calls no allocating routine here.  The array below is part
// of the library's device module: under CUDA's lazy module loading the
// runtime loads that module, and with it reserves the array, on the first
// use of the module on each device -- the first address lookup or launch --
// and that step may allocate device memory and synchronise.  A call with
// C = 0 performs exactly that step (the device check and the address
// lookup) and launches nothing, so a caller can do it ahead of time.  The
// array then lives on that GPU until the process exits.
#include <mutex>
#include <string>

#include "gm_kernels.cuh"

namespace {

// 40 MiB: the per-cell sums, mixture records and projection coefficients,
// the mass-matrix rows and the solver's temporaries of up to kMaxCells cells
// (D = 1 or 3, up to 16 components per cell).
constexpr size_t kScratchBytes = (size_t)40 << 20;
constexpr int64_t kMaxCells = 32768;
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

int fail2(int code, const std::string& msg) { return gmcr::record_error(code, msg.c_str()); }

// Device address of g_scratch on the current device, looked up once per
// device (with that device current).  In host code the symbol is only a
// host-side stand-in; kernels must be given this address.
int scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail2(GM_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail2(GM_ERR_UNSUPPORTED, "device ordinal out of range");
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || !p)
      return fail2(GM_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return GM_OK;
}

}  // namespace

extern "C" {

int gm_reconstruct_noalloc(const gm_config* cfg, int64_t C, const int32_t* K, const double* params,
                           const double* W, const double* rho_target, int64_t n_out,
                           const int64_t* out_off, double* x_out, double* v_out,
                           double* alpha_out, uint32_t* status_out, double* dA_out,
                           void* stream) {
  gmcr::record_error(GM_OK, "");
  int rc = gmcr::api_check_reconstruct(cfg, C, K, params, W, rho_target, n_out, out_off, x_out,
                                       v_out, alpha_out, status_out);
  if (rc) return rc;
  if (C > kMaxCells)
    return fail2(GM_ERR_ARG, "gm_reconstruct_noalloc handles at most 32768 cells per call (got " +
                                 std::to_string((long long)C) + "); use gm_reconstruct");
  if (gmcr::reconstruct_ws_bytes(cfg->D, C, cfg->Kmax) > kScratchBytes)
    return fail2(GM_ERR_ARG, "scratch of gm_reconstruct_noalloc too small for this call");
  if ((rc = gmcr::api_check_device())) return rc;
  void* ws = nullptr;
  if ((rc = scratch_address(&ws))) return rc;  // also the whole of a C = 0 call
  if (C == 0) return GM_OK;
  // every scratch entry a call reads is written earlier in the same call,
  // so nothing has to be cleared between calls
  cudaError_t e = gmcr::launch_reconstruct(cfg->D, C, cfg->Kmax, K, params, W, rho_target, n_out,
                                           out_off, cfg->seed, cfg->L / (double)C, cfg->q,
                                           cfg->shape_order, x_out, v_out, alpha_out, status_out,
                                           dA_out, ws, (cudaStream_t)stream);
  if (e != cudaSuccess) return fail2(GM_ERR_CUDA, std::string("reconstruct launch: ") + cudaGetErrorString(e));
  return GM_OK;
}

// the largest scratch a call may need (kMaxCells cells, 16 components) fits
// the array
int gm_noalloc_limits_ok() {
  return gmcr::reconstruct_ws_bytes(1, kMaxCells, gmcr::kMaxK) <= kScratchBytes &&
         gmcr::reconstruct_ws_bytes(3, kMaxCells, gmcr::kMaxK) <= kScratchBytes;
}

}  // extern "C"
