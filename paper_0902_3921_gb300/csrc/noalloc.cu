// noalloc.cu -- lbm_diagnostics_noalloc: the FP64 diagnostics reduction for
// callers that cannot allocate device memory.
//
// Some callers must not call cudaMalloc: a host framework that owns every
// byte of device memory through its own allocator and budget, or a
// time-critical loop in which cudaMalloc/cudaFree would synchronise the
// device.  This entry point takes the fields from the caller and keeps its
// scratch (the per-block partial sums and the result vector) in the
// file-scope device array below instead of allocating it.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <utility>
#include <vector>

#include "lbm_common.cuh"

namespace hlbm {
cudaError_t launch_diag_raw(const lbm_params &P, double phi0, const double *r_ref,
                            const double *fields, double *partials, int nblocks, double *res,
                            cudaStream_t stream);
}

using namespace hlbm;

namespace {

constexpr int kSitesPerBlock = 2048;  // 256 threads x 8 sites
constexpr size_t kScratchDoubles =
    (size_t)LBM_NOALLOC_MAX_BLOCKS * DIAG_NPART + DIAG_COUNT;

// Loaded with the library on every GPU that uses it and kept until exit:
// partials [LBM_NOALLOC_MAX_BLOCKS][DIAG_NPART] followed by the result vector.
static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

// The device address of a __device__ array belongs to a CUDA context, not to a
// device number: after cudaDeviceReset, or with another context current on
// the same device (a driver-API or green context of a host framework), the
// address must be looked up again.  So the cache is keyed by the current
// context's unique ID (cuCtxGetId), or by its handle where that call is
// missing.
std::mutex g_setup_mutex;
std::vector<std::pair<unsigned long long, double *>> g_scratch_by_ctx;

template <typename F>
F driver_fn(const char *name, int version) {
  void *f = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion(name, &f, version, cudaEnableDefault, &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess)
    return nullptr;
  return reinterpret_cast<F>(f);
}

// key of the context current on this thread; 0 when none is current
unsigned long long current_context_key() {
  static PFN_cuCtxGetCurrent_v4000 get_current = driver_fn<PFN_cuCtxGetCurrent_v4000>("cuCtxGetCurrent", 4000);
  static PFN_cuCtxGetId_v12000 get_id = driver_fn<PFN_cuCtxGetId_v12000>("cuCtxGetId", 12000);
  CUcontext ctx = nullptr;
  if (get_current == nullptr || get_current(&ctx) != CUDA_SUCCESS || ctx == nullptr) return 0;
  unsigned long long id = 0;
  if (get_id != nullptr && get_id(ctx, &id) == CUDA_SUCCESS) return id + 1;
  return static_cast<unsigned long long>(reinterpret_cast<uintptr_t>(ctx));
}

thread_local char g_noalloc_msg[256] = "";

int noalloc_fail(int code, const char *msg) {
  snprintf(g_noalloc_msg, sizeof g_noalloc_msg, "%s", msg);
  return code;
}

}  // namespace

extern "C" {

int lbm_diagnostics_noalloc(const lbm_params *params, const double *fields,
                            const double *r_ref, void *cuda_stream, lbm_diag *out) {
  if (params == nullptr || fields == nullptr || out == nullptr)
    return noalloc_fail(LBM_EINVAL, "lbm_diagnostics_noalloc: NULL argument");
  const lbm_params &P = *params;
  // the checks lbm_create makes, on the fields this function reads
  if ((P.dims != 2 && P.dims != 3) || P.Lx < 3 || P.Ly < 3 || (P.dims == 3 && P.Lz < 3))
    return noalloc_fail(LBM_EINVAL, "lbm_diagnostics_noalloc: bad dims or lattice side < 3");
  if (!std::isfinite(P.a) || !(P.a < 0.0))
    return noalloc_fail(LBM_EINVAL,
                        "lbm_diagnostics_noalloc: a must be finite and < 0 (phi0 = sqrt(-a/b) "
                        "scales the drop area)");
  if (!(P.b > 0.0) || !std::isfinite(P.b))
    return noalloc_fail(LBM_EINVAL, "lbm_diagnostics_noalloc: b must be > 0");
  if (!(P.kappa >= 0.0) || !std::isfinite(P.kappa))
    return noalloc_fail(LBM_EINVAL, "lbm_diagnostics_noalloc: kappa must be >= 0");
  if (!(P.T > 0.0) || !std::isfinite(P.T))
    return noalloc_fail(LBM_EINVAL, "lbm_diagnostics_noalloc: T must be finite and > 0");
  if (!std::isfinite(P.N) || !std::isfinite(P.Q))
    return noalloc_fail(LBM_EINVAL, "lbm_diagnostics_noalloc: N and Q must be finite");
  const long long S = (long long)P.Lx * P.Ly * (P.dims == 3 ? P.Lz : 1);
  if (S > LBM_NOALLOC_MAX_SITES) {
    char buf[200];
    snprintf(buf, sizeof buf,
             "lbm_diagnostics_noalloc: %lld sites exceed the %d-site capacity of its "
             "built-in scratch; use lbm_diagnostics",
             S, LBM_NOALLOC_MAX_SITES);
    return noalloc_fail(LBM_EINVAL, buf);
  }
  double *scratch = nullptr;
  cudaError_t e;
  {
    // once per context, with it current: the device address of the array
    // (its name in host code is only a host-side stand-in)
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    unsigned long long key = current_context_key();
    for (const auto &kv : g_scratch_by_ctx)
      if (key != 0 && kv.first == key) scratch = kv.second;
    if (scratch == nullptr) {
      void *ptr = nullptr;
      e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);  // makes the primary context current if none is
      if (e != cudaSuccess)
        return noalloc_fail(LBM_ECUDA, "lbm_diagnostics_noalloc: cudaGetSymbolAddress failed");
      scratch = static_cast<double *>(ptr);
      if (key == 0) key = current_context_key();
      if (key != 0) {
        for (auto &kv : g_scratch_by_ctx)
          if (kv.first == key) kv.second = scratch, key = 0;
        if (key != 0) g_scratch_by_ctx.emplace_back(key, scratch);
      }
    }
  }
  const int nblocks = (int)((S + kSitesPerBlock - 1) / kSitesPerBlock);
  const double centre[3] = {P.Lx / 2.0, P.Ly / 2.0, P.dims == 3 ? P.Lz / 2.0 : 0.0};
  const double *rr = r_ref ? r_ref : centre;
  const double ref3[3] = {rr[0], rr[1], P.dims == 3 ? rr[2] : 0.0};
  const double phi0 = std::sqrt(-P.a / P.b);
  cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
  double *partials = scratch;
  double *res = scratch + (size_t)LBM_NOALLOC_MAX_BLOCKS * DIAG_NPART;
  // every partial slot and result entry read below is written earlier in
  // this call, so nothing has to be cleared between calls
  e = launch_diag_raw(P, phi0, ref3, fields, partials, nblocks, res, stream);
  if (e != cudaSuccess) return noalloc_fail(LBM_ECUDA, cudaGetErrorString(e));
  double host[DIAG_COUNT];
  e = cudaMemcpyAsync(host, res, sizeof host, cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) return noalloc_fail(LBM_ECUDA, cudaGetErrorString(e));
  memset(out, 0, sizeof *out);
  out->t = -1;
  out->sum_n = host[DIAG_SUM_N];
  out->sum_phi = host[DIAG_SUM_PHI];
  out->u_max = host[DIAG_UMAX];
  out->dp = host[DIAG_DP];
  out->area = host[DIAG_AREA];
  out->R_eff = P.dims == 2 ? std::sqrt(out->area / M_PI) : std::cbrt(3.0 * out->area / (4.0 * M_PI));
  out->nonfinite = host[DIAG_NONFINITE] != 0.0;
  for (int k = 0; k < P.dims; k++) {
    out->momentum[k] = host[DIAG_MOM0 + k];
    out->r_cm[k] = host[DIAG_RCM0 + k];
    out->v_f[k] = host[DIAG_VF0 + k];
  }
  g_noalloc_msg[0] = '\0';
  return out->nonfinite ? LBM_ENONFINITE : LBM_OK;
}

const char *lbm_noalloc_last_error(void) { return g_noalloc_msg; }

}  // extern "C"
