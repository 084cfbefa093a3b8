// noalloc.cu -- lbm_diagnostics_noalloc: the FP64 diagnostics reduction for
// callers that cannot allocate device memory.
//
// Some callers must not call cudaMalloc: a host framework that owns every
// byte of device memory through its own allocator and budget, or a
// time-critical loop in which cudaMalloc/cudaFree would synchronise the
// device.  This entry point takes the fields from the caller and keeps its
// scratch (the per-block partial sums and the result vector) in the
// file-scope device array below instead of allocating it.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>

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

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
double *g_scratch_ptr[kMaxDevices] = {nullptr};

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
  if ((P.dims != 2 && P.dims != 3) || P.Lx < 3 || P.Ly < 3 || (P.dims == 3 && P.Lz < 3))
    return noalloc_fail(LBM_EINVAL, "lbm_diagnostics_noalloc: bad dims or lattice side < 3");
  if (!(P.b > 0.0))
    return noalloc_fail(LBM_EINVAL, "lbm_diagnostics_noalloc: b must be > 0");
  const long long S = (long long)P.Lx * P.Ly * (P.dims == 3 ? P.Lz : 1);
  if (S > LBM_NOALLOC_MAX_SITES) {
    char buf[200];
    snprintf(buf, sizeof buf,
             "lbm_diagnostics_noalloc: %lld sites exceed the %d-site capacity of its "
             "built-in scratch; use lbm_diagnostics",
             S, LBM_NOALLOC_MAX_SITES);
    return noalloc_fail(LBM_EINVAL, buf);
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return noalloc_fail(LBM_ECUDA, "lbm_diagnostics_noalloc: no usable current device");
  double *scratch;
  {
    // once per device, with that device current: the device address of the
    // array (its name in host code is only a host-side stand-in)
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (g_scratch_ptr[dev] == nullptr) {
      void *ptr = nullptr;
      e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
      if (e != cudaSuccess)
        return noalloc_fail(LBM_ECUDA, "lbm_diagnostics_noalloc: cudaGetSymbolAddress failed");
      g_scratch_ptr[dev] = static_cast<double *>(ptr);
    }
    scratch = g_scratch_ptr[dev];
  }
  const int nblocks = (int)((S + kSitesPerBlock - 1) / kSitesPerBlock);
  const double centre[3] = {P.Lx / 2.0, P.Ly / 2.0, P.dims == 3 ? P.Lz / 2.0 : 0.0};
  const double *rr = r_ref ? r_ref : centre;
  const double ref3[3] = {rr[0], rr[1], P.dims == 3 ? rr[2] : 0.0};
  const double phi0 = P.a < 0 ? std::sqrt(-P.a / P.b) : 1.0;
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
