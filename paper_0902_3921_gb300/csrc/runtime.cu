// runtime.cu -- the C ABI of include/hybrid_lbm.h: validation, the choice of
// the FD substep count (Sec. II C), device allocation, the per-step launch
// sequence (captured into CUDA graphs), kernel timing, FP64 read-back and
// checkpoints.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>

#include "lbm_common.cuh"

namespace hlbm {

cudaError_t collide2d_launch(lbm_handle *h, int in, int force_on, int mode);
cudaError_t fd2d_launch(lbm_handle *h, int in);
cudaError_t density2d_launch(lbm_handle *h, int in);
cudaError_t collide2d_configure(int precision);
cudaError_t collide3d_launch(lbm_handle *h, int in, int force_on, int mode);
cudaError_t fd3d_launch(lbm_handle *h, int in);
cudaError_t density3d_launch(lbm_handle *h, int in);
size_t fd3d_smem_bytes(int precision, int sub);
cudaError_t fd3d_configure(int precision, size_t smem);

template <typename C>
KParams<C> make_params(const lbm_handle *h, int force_on) {
  const lbm_params &P = h->P;
  KParams<C> p;
  p.Lx = P.Lx;
  p.Ly = P.Ly;
  p.Lz = h->dims == 3 ? P.Lz : 1;
  p.a = (C)P.a;
  p.b = (C)P.b;
  p.kappa = (C)P.kappa;
  p.tau_inv = (C)(1.0 / P.tau);
  p.pref = (C)(1.0 - 1.0 / (2.0 * P.tau));
  p.N = (C)P.N;
  p.Q = (C)P.Q;
  if (h->dims == 2) {
    p.M = (C)((1.0 - 2.0 * P.N) / 4.0);
    p.R = (C)((1.0 - P.Q) / 2.0);
    p.C0 = (C)(-4.0 * (P.Q + (1.0 - P.Q) / 2.0));
  } else {
    p.M = (C)((1.0 - 2.0 * P.N) / 8.0);
    p.R = (C)((1.0 - P.Q) / 4.0);
    p.C0 = (C)(-(6.0 * P.Q + 12.0 * (1.0 - P.Q) / 4.0));
  }
  p.gx = force_on ? (C)P.g[0] : C(0);
  p.gy = force_on ? (C)P.g[1] : C(0);
  p.gz = (force_on && h->dims == 3) ? (C)P.g[2] : C(0);
  p.cs2mT = (C)(1.0 / 3.0 - P.T);
  p.dt = (C)(1.0 / h->m);
  p.dtG = (C)(P.Gamma / h->m);
  if (P.precision == LBM_F16DEV) {
    p.scale = (C)std::ldexp(1.0, P.f16_scale_log2);
    p.inv_scale = (C)std::ldexp(1.0, -P.f16_scale_log2);
  } else {
    p.scale = C(1);
    p.inv_scale = C(1);
  }
  p.adv_variant = P.adv_variant;
  p.cubic_at_half = P.cubic_at_half;
  p.stencil_fd = P.stencil_fd;
  return p;
}
template KParams<float> make_params<float>(const lbm_handle *, int);
template KParams<double> make_params<double>(const lbm_handle *, int);

cudaError_t launch_collide(lbm_handle *h, int in, int force_on, int mode) {
  return h->dims == 2 ? collide2d_launch(h, in, force_on, mode)
                      : collide3d_launch(h, in, force_on, mode);
}
cudaError_t launch_fd(lbm_handle *h, int in) {
  return h->dims == 2 ? fd2d_launch(h, in) : fd3d_launch(h, in);
}
cudaError_t launch_density(lbm_handle *h, int in) {
  return h->dims == 2 ? density2d_launch(h, in) : density3d_launch(h, in);
}

}  // namespace hlbm

using namespace hlbm;

namespace {

thread_local std::string g_create_error;
constexpr int kGraphChunk = 64;        // LB steps per captured graph (even)
constexpr size_t kMaxGraphs = 16;      // graph cache entries per handle
constexpr size_t kMaxEventPairs = 8192;

int fail(lbm_handle *h, int code, const std::string &msg) {
  if (h == nullptr) {
    g_create_error = msg;
  } else if (h->err == 0) {
    h->err = code;
    h->msg = msg;
  }
  return code;
}

// A refusal that leaves the handle usable: the text is kept for
// lbm_last_error, nothing is latched.
int refuse(lbm_handle *h, int code, const std::string &msg) {
  if (h->err == 0) h->msg = msg;
  return code;
}

int cuda_fail(lbm_handle *h, cudaError_t e, const char *what) {
  return fail(h, e == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA,
              std::string(what) + ": " + cudaGetErrorString(e));
}

// After a synchronisation: a bounded device wait of the TMA collide kernel
// that gave up (its copies never completed) latches LBM_ETIMEOUT.
int check_device_waits(lbm_handle *h) {
  if (h->tma_ready && collide2d_tma_error(true) > 0)
    return fail(h, LBM_ETIMEOUT, "collide kernel: a TMA copy did not complete within its wait bound");
  if (h->dims == 3 && h->P.precision != LBM_F64 && fd3p_error(true) > 0)
    return fail(h, LBM_ETIMEOUT, "FD substep kernel: a bulk copy did not complete within its wait bound");
  return LBM_OK;
}

#define CK(h, call, what)                              \
  do {                                                 \
    cudaError_t e_ = (call);                           \
    if (e_ != cudaSuccess) return cuda_fail(h, e_, what); \
  } while (0)

size_t storage_bytes(int precision) {
  return precision == LBM_F64 ? 8 : (precision == LBM_F32DEV ? 4 : 2);
}
size_t compute_bytes(int precision) { return precision == LBM_F64 ? 8 : 4; }

// Stiffness of the diffusive half step (Eq. 36) at the checkerboard mode:
// Gamma (a_eff lam + kappa lam^2), lam = 4 d the largest eigenvalue of the
// 5-point (7-point) Laplacian and a_eff = a + 3 b phi0^2 = -2a in the ordered
// phase (a < 0), a otherwise.
// Largest eigenvalue lam of -lap over the Brillouin zone: 4 d for the 5/7-point
// Laplacian; for lap_D of Eq. 31 (stencil_fd, 2D) the symbol 4(Q + R) -
// 2Q (cos kx + cos ky) - 4R cos kx cos ky is bilinear in the cosines, so its
// maximum is at a corner: max(8Q, 4).
double fd_stiffness(const lbm_params &P) {
  const double lam = (P.stencil_fd && P.dims == 2) ? std::max(8.0 * P.Q, 4.0) : 4.0 * P.dims;
  const double aeff = P.a < 0 ? -2.0 * P.a : P.a;
  return P.Gamma * (aeff * lam + P.kappa * lam * lam);
}

// Host-side fault injection for testing the error paths (LBM_FAULT):
// "alloc" refuses lbm_create as if the first device allocation failed, before
// any CUDA call; "alloc:K" fails the K-th allocation (the earlier ones are
// freed again); "h2d" fails the host-to-device copy of lbm_init_fields.
// Returns the allocation index to fail (0: before any call, -1: none) for
// "alloc", and sets *h2d for "h2d".
int injected_fault(bool *h2d) {
  *h2d = false;
  const char *f = std::getenv("LBM_FAULT");
  if (f == nullptr) return -1;
  if (std::strcmp(f, "h2d") == 0) {
    *h2d = true;
    return -1;
  }
  if (std::strcmp(f, "alloc") == 0) return 0;
  int k = 0;
  if (std::sscanf(f, "alloc:%d", &k) == 1 && k >= 1) return k;
  return -1;
}

int validate(const lbm_params *P, std::string &why) {
  if (P == nullptr) return why = "params is NULL", LBM_EINVAL;
  if (P->dims != 2 && P->dims != 3) return why = "dims must be 2 or 3", LBM_EINVAL;
  if (P->Lx < 3 || P->Ly < 3 || (P->dims == 3 && P->Lz < 3))
    return why = "every lattice side must be >= 3", LBM_EINVAL;
  const long long S = (long long)P->Lx * P->Ly * (P->dims == 3 ? P->Lz : 1);
  if (S > (1LL << 31)) return why = "more than 2^31 sites", LBM_EINVAL;
  if (!(P->tau > 0.5) || !std::isfinite(P->tau)) return why = "tau must be > 1/2", LBM_EINVAL;
  if (!(P->b > 0.0) || !std::isfinite(P->b)) return why = "b must be > 0", LBM_EINVAL;
  if (!(P->kappa >= 0.0) || !std::isfinite(P->kappa)) return why = "kappa must be >= 0", LBM_EINVAL;
  if (!(P->Gamma >= 0.0) || !std::isfinite(P->Gamma)) return why = "Gamma must be >= 0", LBM_EINVAL;
  if (!std::isfinite(P->a) || !std::isfinite(P->T) || !(P->T > 0.0))
    return why = "a must be finite and T > 0", LBM_EINVAL;
  if (!std::isfinite(P->N) || !std::isfinite(P->Q)) return why = "N and Q must be finite", LBM_EINVAL;
  for (int k = 0; k < 3; k++)
    if (!std::isfinite(P->g[k])) return why = "g must be finite", LBM_EINVAL;
  if (P->force_steps < 0) return why = "force_steps must be >= 0", LBM_EINVAL;
  if (P->precision != LBM_F64 && P->precision != LBM_F32DEV && P->precision != LBM_F16DEV)
    return why = "unknown precision", LBM_EINVAL;
  if (P->adv_variant != LBM_ADV_PAPER && P->adv_variant != LBM_ADV_FLUX)
    return why = "unknown adv_variant", LBM_EINVAL;
  if (P->f16_scale_log2 < 0 || P->f16_scale_log2 > 14)
    return why = "f16_scale_log2 must be in 0..14", LBM_EINVAL;
  if (std::abs(P->fd_substeps) > 4096) return why = "fd_substeps too large", LBM_EINVAL;
  if (P->stencil_fd != 0 && P->stencil_fd != 1) return why = "stencil_fd must be 0 or 1", LBM_EINVAL;
  if (P->stencil_fd && (P->dims != 2 || P->adv_variant != LBM_ADV_PAPER))
    return why = "stencil_fd is a 2D option of the printed advection form", LBM_EINVAL;
  if (P->stencil_fd && !(P->Q >= 0.0))
    return why = "stencil_fd needs Q >= 0 (lap_D is otherwise not negative semi-definite)", LBM_EINVAL;
  return LBM_OK;
}

void harvest_events(lbm_handle *h) {
  if (h->events.empty()) return;
  cudaStreamSynchronize(h->stream);
  for (auto &ev : h->events) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, ev.a, ev.b) == cudaSuccess) {
      h->ms_acc[ev.family] += ms;
      h->launches_acc[ev.family] += 1;
    }
    cudaEventDestroy(ev.a);
    cudaEventDestroy(ev.b);
  }
  h->events.clear();
}

// Runs one kernel family, bracketed by events when timing is on.
template <typename F>
int timed(lbm_handle *h, int family, F &&launch, const char *what) {
  if (!h->timing) {
    CK(h, launch(), what);
    return LBM_OK;
  }
  if (h->events.size() >= kMaxEventPairs) harvest_events(h);
  EventPair ev;
  ev.family = family;
  CK(h, cudaEventCreate(&ev.a), "cudaEventCreate");
  CK(h, cudaEventCreate(&ev.b), "cudaEventCreate");
  CK(h, cudaEventRecord(ev.a, h->stream), "cudaEventRecord");
  CK(h, launch(), what);
  CK(h, cudaEventRecord(ev.b, h->stream), "cudaEventRecord");
  h->events.push_back(ev);
  return LBM_OK;
}

// One hybrid step queued on the stream: (density), collide/stream, FD update.
int queue_step(lbm_handle *h, int force_on) {
  const int in = h->cur;
  int rc;
  if (h->P.T != 1.0 / 3.0) {
    rc = timed(h, 2, [&] { return launch_density(h, in); }, "density kernel");
    if (rc) return rc;
  }
  rc = timed(h, 0, [&] { return launch_collide(h, in, force_on, COLLIDE_STEP); },
             "collide kernel");
  if (rc) return rc;
  rc = timed(h, 1, [&] { return launch_fd(h, in); }, "FD kernel");
  if (rc) return rc;
  h->cur = 1 - in;
  h->t += 1;
  return LBM_OK;
}

int run_graph(lbm_handle *h, long long nsteps, int force_on) {
  const int parity = h->cur;
  cudaGraphExec_t exec = nullptr;
  for (auto &g : h->graphs)
    if (g.nsteps == nsteps && g.parity == parity && g.force_on == force_on) exec = g.exec;
  if (exec == nullptr) {
    const long long t0 = h->t;
    CK(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal),
       "cudaStreamBeginCapture");
    int rc = LBM_OK;
    for (long long k = 0; k < nsteps && rc == LBM_OK; k++) rc = queue_step(h, force_on);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(h->stream, &graph);
    h->cur = parity;  // capture only recorded the launches
    h->t = t0;
    if (rc) return rc;
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaGraphInstantiate");
    if (h->graphs.size() >= kMaxGraphs) {
      cudaGraphExecDestroy(h->graphs.front().exec);
      h->graphs.erase(h->graphs.begin());
    }
    h->graphs.push_back(GraphEntry{nsteps, parity, force_on, exec});
  }
  CK(h, cudaGraphLaunch(exec, h->stream), "cudaGraphLaunch");
  if (nsteps % 2) h->cur = 1 - h->cur;
  h->t += nsteps;
  return LBM_OK;
}

int run_segment(lbm_handle *h, long long len, int force_on) {
  if (!h->use_graphs || h->timing) {
    for (long long k = 0; k < len; k++) {
      int rc = queue_step(h, force_on);
      if (rc) return rc;
    }
    return LBM_OK;
  }
  while (len > 0) {
    const long long chunk = std::min<long long>(len, kGraphChunk);
    int rc = run_graph(h, chunk, force_on);
    if (rc) return rc;
    len -= chunk;
  }
  return LBM_OK;
}

int check_usable(lbm_handle *h, bool need_init) {
  if (h == nullptr) return LBM_EINVAL;
  if (h->err) return h->err;
  if (need_init && !h->inited) return fail(h, LBM_ESTATE, "fields are not initialised");
  return LBM_OK;
}

// n(t), phi(t), u*(t) as FP64 in staging.
int queue_moments(lbm_handle *h) {
  if (h->P.T != 1.0 / 3.0) CK(h, launch_density(h, h->cur), "density kernel");
  CK(h, launch_collide(h, h->cur, h->t < h->P.force_steps, COLLIDE_MOMENTS), "moments kernel");
  return LBM_OK;
}

uint32_t crc32_update(uint32_t crc, const unsigned char *p, size_t n) {
  // CRC-32 (IEEE 802.3, reflected polynomial 0xEDB88320), bitwise
  crc = ~crc;
  for (size_t i = 0; i < n; i++) {
    crc ^= p[i];
    for (int k = 0; k < 8; k++) crc = (crc >> 1) ^ (0xEDB88320u & (0u - (crc & 1u)));
  }
  return ~crc;
}

struct CkptHeader {
  char magic[8];
  uint32_t version;
  uint32_t crc;
  long long t;
  long long payload;
  lbm_params P;
};

bool same_params(const lbm_params &a, const lbm_params &b) {
  return a.dims == b.dims && a.Lx == b.Lx && a.Ly == b.Ly && (a.dims == 2 || a.Lz == b.Lz) &&
         a.a == b.a && a.b == b.b && a.kappa == b.kappa && a.T == b.T && a.tau == b.tau &&
         a.Gamma == b.Gamma && a.N == b.N && a.Q == b.Q && a.fd_substeps == b.fd_substeps &&
         a.adv_variant == b.adv_variant && a.cubic_at_half == b.cubic_at_half &&
         a.g[0] == b.g[0] && a.g[1] == b.g[1] && a.g[2] == b.g[2] &&
         a.force_steps == b.force_steps && a.precision == b.precision && a.stencil_fd == b.stencil_fd &&
         a.f16_scale_log2 == b.f16_scale_log2;
}

// Times fn() (three launches after one warm-up) with CUDA events on the
// handle's stream; returns milliseconds or a negative value on error.
template <typename F>
float time_launches(lbm_handle *h, cudaEvent_t e0, cudaEvent_t e1, F &&fn) {
  cudaError_t e = fn();
  float ms = -1.f;
  if (e == cudaSuccess) e = cudaEventRecord(e0, h->stream);
  for (int k = 0; k < 3 && e == cudaSuccess; k++) e = fn();
  if (e == cudaSuccess) e = cudaEventRecord(e1, h->stream);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  return e == cudaSuccess ? ms : -1.f;
}

// Autotuner of the 2D launch shapes, timed with CUDA events on the handle's
// own (zeroed) buffers: for the FD kernel the columns per lane (FP32: 2 or
// 4), the substeps per launch (<= 4) and the output rows per warp; for the
// collide kernel the sites per thread (2 or 4).
int autotune_2d(lbm_handle *h) {
  if (const char *fixed = std::getenv("HLBM_TUNING")) {
    int v[5] = {h->sub, h->fd_rows, h->fd_cols, h->collide_rows, 0};
    const int nv = std::sscanf(fixed, "%d,%d,%d,%d,%d", &v[0], &v[1], &v[2], &v[3], &v[4]);
    // block kernel shapes: sub, region rows, warps / 8
    const int shapes[7][3] = {{1, 64, 2}, {2, 64, 2}, {2, 80, 2}, {4, 80, 2}, {4, 96, 2}, {4, 96, 4}, {2, 96, 4}};
    bool block_ok = false;
    for (const auto &sh : shapes)
      block_ok |= v[4] == 128 && h->P.precision != LBM_F64 && v[0] == sh[0] && v[1] == sh[1] && v[2] == sh[2];
    // wavefront kernel: 2 or 4 substeps per launch, rows = output rows of a segment
    const bool wave_ok = v[4] == 1 && fd2d_wave_eligible(h) && (std::min(v[0], h->m) == 2 || std::min(v[0], h->m) == 4);
    if (nv == 5 && v[4] == 1 && !wave_ok) {
      return fail(h, LBM_EINVAL,
                  "HLBM_TUNING wavefront FD kernel (tile 1): sub 2 or 4 (m >= 2), FP32 or FP16 storage, "
                  "printed advection form, Lx % 4 == 0");
    }
    if (h->P.stencil_fd && !(nv == 5 && (v[4] == 32 || v[4] == 64)))
      return fail(h, LBM_EINVAL, "HLBM_TUNING: stencil_fd runs on the tile FD kernel (tile 32 or 64)");
    if ((nv == 4 || (nv == 5 && (v[4] == 0 || v[4] == 32 || v[4] == 64 || block_ok || wave_ok))) && v[0] >= 1 &&
        v[0] <= 4 && v[1] >= 1 && (v[2] == 2 || v[2] == 4) &&
        (v[3] == 2 || v[3] == 4 || (v[3] <= 1 && v[3] >= 0 && h->P.precision != LBM_F16DEV) ||
         collide2d_tma_eligible(h, v[3]))) {
      h->sub = std::min(v[0], h->m);
      h->fd_rows = v[1];
      h->fd_cols = h->P.precision == LBM_F64 ? 2 : v[2];
      h->collide_rows = v[3];
      h->fd_tile_w = v[4];
      if (h->fd_tile_w == 32) h->sub = 1;
      if (h->fd_tile_w == 64) h->sub = std::min(h->sub, 2);
      return LBM_OK;
    }
    if (nv == 5 && v[4] == 128 && !block_ok) {
      return fail(h, LBM_EINVAL,
                  "HLBM_TUNING block kernel shapes (sub,rows,cols): (1,64,2) (2,64,2) (2,80,2) (4,80,2) "
                  "(4,96,2) (4,96,4) (2,96,4), FP32 only");
    }
    return fail(h, LBM_EINVAL, "HLBM_TUNING must be 'sub,rows,cols,collide_rows[,tile]'");
  }
  // one choice per lattice shape and scheme in a process: every handle of
  // the same problem then runs the same kernels (and gives the same bits)
  using Key = std::tuple<int, int, int, int, int, int, int>;
  struct Choice {
    int sub, fd_rows, fd_cols, collide_rows, fd_tile_w;
  };
  static std::mutex cache_mu;
  static std::map<Key, Choice> cache;
  int dev = 0;
  cudaGetDevice(&dev);
  const Key key{dev, h->P.Lx, h->P.Ly, h->P.precision, h->m, h->P.adv_variant, h->P.cubic_at_half};
  {
    std::lock_guard<std::mutex> lk(cache_mu);
    auto it = cache.find(key);
    if (it != cache.end()) {
      h->sub = it->second.sub;
      h->fd_rows = it->second.fd_rows;
      h->fd_cols = it->second.fd_cols;
      h->collide_rows = it->second.collide_rows;
      h->fd_tile_w = it->second.fd_tile_w;
      return LBM_OK;
    }
  }
  const bool verbose = std::getenv("HLBM_TUNE_VERBOSE") != nullptr;
  const size_t cb = compute_bytes(h->P.precision);
  CK(h, cudaMemsetAsync(h->phi[0], 0, cb * (size_t)h->S, h->stream), "cudaMemset");
  CK(h, cudaMemsetAsync(h->u, 0, cb * h->dims * (size_t)h->S, h->stream), "cudaMemset");
  CK(h, cudaMemsetAsync(h->h[0], 0, h->hbytes, h->stream), "cudaMemset");
  struct FdShape {
    int tile_w, cols, sub, rows;
  };
  std::vector<FdShape> cands;
  const bool stencil = h->P.stencil_fd != 0;  // only the tile kernel evaluates the stencil operators
  // wavefront kernel (FP32 phi): 128-column strips marching down segments of
  // `rows` output rows, 4 or 2 substeps per launch
  // (one CTA marches a whole segment, so the segment heights offered are the
  // ones that make the grid one to eight whole waves of resident CTAs)
  if (fd2d_wave_eligible(h) && !stencil) {
    for (int sb : {4, 2}) {
      if (sb > h->m) continue;
      int strips = 1;
      const int slots = fd2d_wave_slots(sb, &strips, h->P.Lx);
      std::vector<int> nys;
      for (int w = 1; w <= 8 && slots > 0; w++) {
        const int spp = w * slots / strips;  // segments per strip
        if (spp < 1) continue;
        const int ny = (h->P.Ly + spp - 1) / spp;
        if (ny >= 8 && std::find(nys.begin(), nys.end(), ny) == nys.end()) nys.push_back(ny);
      }
      if (nys.empty()) nys.push_back(std::min(h->P.Ly, 64));
      for (int ny : nys) cands.push_back({1, 4, sb, ny});
    }
  }
  // block kernel (FP32): 128-column regions, (substeps, rows per warp)
  if (h->P.precision != LBM_F64 && !stencil) {
    if (h->m >= 4) {
      cands.push_back({128, 2, 4, 80});
      cands.push_back({128, 2, 4, 96});
      cands.push_back({128, 4, 4, 96});
    }
    if (h->m >= 2) {
      cands.push_back({128, 2, 2, 64});
      cands.push_back({128, 2, 2, 80});
      cands.push_back({128, 4, 2, 96});
    }
    cands.push_back({128, 2, 1, 64});
  }
  // shared-memory tile kernel: 64 wide with 1 or 2 substeps, 32 wide with 1
  cands.push_back({32, 4, 1, 32});
  cands.push_back({64, 4, 1, 32});
  if (h->m >= 2) cands.push_back({64, 4, 2, 32});
  // warp-marching kernel: columns per lane, substeps per launch, rows per warp
  const int subs[3] = {std::min(h->m, 4), std::min(h->m, 2), 1};
  const int rows[5] = {8, 16, 32, 64, 128};
  for (int cols : {4, 2}) {
    if (stencil) break;
    if (cols == 4 && h->P.precision == LBM_F64) continue;
    for (int si = 0; si < 3; si++) {
      if (si > 0 && subs[si] == subs[si - 1]) continue;
      for (int ri = 0; ri < 5; ri++) {
        if (ri > 0 && rows[ri - 1] >= h->P.Ly) break;  // taller tiles change nothing
        cands.push_back({0, cols, subs[si], rows[ri]});
      }
    }
  }
  cudaEvent_t e0, e1;
  CK(h, cudaEventCreate(&e0), "cudaEventCreate");
  CK(h, cudaEventCreate(&e1), "cudaEventCreate");
  float best = 1e30f;
  FdShape bestc = cands[0];
  for (const FdShape &c : cands) {
    h->fd_tile_w = c.tile_w;
    h->fd_cols = c.cols;
    h->sub = c.sub;
    h->fd_rows = c.rows;
    const float ms = time_launches(h, e0, e1, [&] { return launch_fd(h, 0); });
    if (verbose)
      std::fprintf(stderr, "hlbm tune fd %dx%d tile=%d cols=%d sub=%d rows=%d: %.1f us\n",
                   h->P.Lx, h->P.Ly, c.tile_w, c.cols, c.sub, c.rows, ms * 1000.f / 3);
    if (ms < 0) {
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      return cuda_fail(h, cudaGetLastError(), "FD autotuning");
    }
    if (ms < best) {
      best = ms;
      bestc = c;
    }
  }
  h->fd_tile_w = bestc.tile_w;
  h->fd_cols = bestc.cols;
  h->sub = bestc.sub;
  h->fd_rows = bestc.rows;
  best = 1e30f;
  int best_cr = 2;
  for (int cr : {0, 1, 2, 4, 3, 5, 6, 7}) {
    if (cr < 2 && h->P.precision == LBM_F16DEV) continue;  // cp.async moves >= 4 bytes
    if ((cr >= 5 || cr == 3) && !collide2d_tma_eligible(h, cr)) continue;
    h->collide_rows = cr;
    const float ms =
        time_launches(h, e0, e1, [&] { return launch_collide(h, 0, 0, COLLIDE_STEP); });
    if (verbose)
      std::fprintf(stderr, "hlbm tune collide %dx%d rows=%d: %.1f us\n", h->P.Lx, h->P.Ly, cr,
                   ms * 1000.f / 3);
    if (ms < 0) {
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      return cuda_fail(h, cudaGetLastError(), "collide autotuning");
    }
    if (ms < best) {
      best = ms;
      best_cr = cr;
    }
  }
  h->collide_rows = best_cr;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  std::lock_guard<std::mutex> lk(cache_mu);
  cache.emplace(key, Choice{h->sub, h->fd_rows, h->fd_cols, h->collide_rows, h->fd_tile_w});
  return LBM_OK;
}

}  // namespace

namespace hlbm {
// Off unless HLBM_PDL=1: measured on GB300, the early-scheduled dependent
// grids made the graph-timed step slower, not faster (4096^2 FP32: 48.6
// against 53.8 GLUPS; the 512-drop batch: 464 against 362 us per step).
bool pdl_enabled() {
  static const bool on = [] {
    const char *e = std::getenv("HLBM_PDL");
    return e && e[0] == '1';
  }();
  return on;
}

// n(t), phi(t), u*(t) as FP64 in the handle's staging buffer (surrogate coupling)
int queue_moments_for(lbm_handle *h) { return queue_moments(h); }
}  // namespace hlbm

extern "C" {

int lbm_lattice(int dims, int *e, double *w) {
  if (dims != 2 && dims != 3) return LBM_EINVAL;
  const int q = dims == 2 ? 9 : 19;
  for (int i = 0; i < q; i++) {
    if (e) {
      e[3 * i + 0] = dims == 2 ? q9_ex(i) : q19_ex(i);
      e[3 * i + 1] = dims == 2 ? q9_ey(i) : q19_ey(i);
      e[3 * i + 2] = dims == 2 ? 0 : q19_ez(i);
    }
    if (w) w[i] = dims == 2 ? q9_w(i) : q19_w(i);
  }
  return q;
}

int lbm_buffer_bytes(const lbm_params *params, unsigned long long bytes[3]) {
  if (bytes == nullptr) return fail(nullptr, LBM_EINVAL, "bytes is NULL");
  std::string why;
  int rc = validate(params, why);
  if (rc) return fail(nullptr, rc, why);
  const unsigned long long S =
      (unsigned long long)params->Lx * params->Ly * (params->dims == 3 ? params->Lz : 1);
  const int q = params->dims == 2 ? 9 : 19;
  bytes[0] = storage_bytes(params->precision) * q * S;
  bytes[1] = compute_bytes(params->precision) * S;
  bytes[2] = compute_bytes(params->precision) * params->dims * S;
  return LBM_OK;
}

static int create_impl(const lbm_params *params, void *cuda_stream, const lbm_buffers *adopt,
                       lbm_handle **out);

int lbm_create(const lbm_params *params, void *cuda_stream, lbm_handle **out) {
  return create_impl(params, cuda_stream, nullptr, out);
}

int lbm_create_with_buffers(const lbm_params *params, void *cuda_stream, const lbm_buffers *buffers,
                            lbm_handle **out) {
  if (out) *out = nullptr;
  if (buffers == nullptr) return fail(nullptr, LBM_EINVAL, "buffers is NULL");
  const void *ptrs[6] = {buffers->populations[0], buffers->populations[1], buffers->phi[0],
                         buffers->phi[1], buffers->phi[2], buffers->u};
  for (const void *q : ptrs)
    if (q == nullptr || reinterpret_cast<uintptr_t>(q) % 16 != 0)
      return fail(nullptr, LBM_EINVAL, "every lbm_buffers pointer must be non-NULL and 16-byte aligned");
  return create_impl(params, cuda_stream, buffers, out);
}

static int create_impl(const lbm_params *params, void *cuda_stream, const lbm_buffers *adopt,
                       lbm_handle **out) {
  if (out == nullptr) return fail(nullptr, LBM_EINVAL, "out is NULL");
  *out = nullptr;
  std::string why;
  int rc = validate(params, why);
  if (rc) return fail(nullptr, rc, why);
  bool fault_h2d = false;
  const int fault_alloc = injected_fault(&fault_h2d);
  if (fault_alloc == 0)
    return fail(nullptr, LBM_ENOMEM, "injected fault (LBM_FAULT=alloc): device allocation refused");
  lbm_params P = *params;
  if (P.dims == 2) P.Lz = 1;
  if (P.precision == LBM_F16DEV && P.f16_scale_log2 == 0) P.f16_scale_log2 = 10;
  const double stiff = fd_stiffness(P);
  const int m_min = std::max(1, (int)std::ceil(stiff / 2.0 - 1e-12));
  int m;
  if (P.fd_substeps == 0) {
    m = std::max(1, (int)std::ceil(stiff / 1.5 - 1e-12));
  } else if (P.fd_substeps > 0) {
    m = P.fd_substeps;
    if (m < m_min) {
      char buf[160];
      std::snprintf(buf, sizeof buf,
                    "fd_substeps = %d is below the explicit-Euler bound m >= %d of the "
                    "diffusive step (pass -m to force it)",
                    m, m_min);
      return fail(nullptr, LBM_EINVAL, buf);
    }
  } else {
    m = -P.fd_substeps;
  }
  lbm_handle *h = new lbm_handle();
  h->P = P;
  h->dims = P.dims;
  h->q = P.dims == 2 ? 9 : 19;
  h->m = m;
  h->S = (long long)P.Lx * P.Ly * P.Lz;
  h->phi0 = P.a < 0 ? std::sqrt(-P.a / P.b) : 1.0;
  h->sub = std::min(m, P.dims == 2 ? 4 : 1);
  h->r_ref[0] = P.Lx / 2.0;
  h->r_ref[1] = P.Ly / 2.0;
  h->r_ref[2] = P.dims == 3 ? P.Lz / 2.0 : 0.0;
  auto bail = [&](int code) {
    g_create_error = h->msg;
    lbm_free(h);
    return code;
  };
  if (cuda_stream) {
    h->stream = static_cast<cudaStream_t>(cuda_stream);
  } else {
    cudaError_t e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return bail(cuda_fail(h, e, "cudaStreamCreate"));
    h->own_stream = true;
  }
  const size_t sb = storage_bytes(P.precision), cb = compute_bytes(P.precision);
  h->hbytes = sb * h->q * (size_t)h->S;
  h->phibytes = cb * (size_t)h->S;
  struct {
    void **p;
    size_t n;
  } allocs[] = {{&h->h[0], h->hbytes},
                {&h->h[1], h->hbytes},
                {&h->phi[0], h->phibytes},
                {&h->phi[1], h->phibytes},
                {&h->phi[2], h->phibytes},
                {&h->u, cb * h->dims * (size_t)h->S},
                {(void **)&h->staging, sizeof(double) * (h->dims + 3) * (size_t)h->S},
                {(void **)&h->partials, sizeof(double) * DIAG_BLOCKS * DIAG_NPART},
                {(void **)&h->dres, sizeof(double) * DIAG_COUNT},
                {&h->dn, P.T != 1.0 / 3.0 ? cb * (size_t)h->S : 0},
                {&h->fd_a, h->dims == 3 && P.precision != LBM_F64 ? h->phibytes : 0},
                {&h->fd_p, h->dims == 3 && P.precision != LBM_F64 ? h->phibytes : 0},
                {(void **)&h->sched, h->dims == 2 && P.precision == LBM_F32DEV ? 2 * sizeof(unsigned) : 0}};
  if (adopt) {
    h->adopted = true;
    h->h[0] = adopt->populations[0];
    h->h[1] = adopt->populations[1];
    for (int k = 0; k < 3; k++) h->phi[k] = adopt->phi[k];
    h->u = adopt->u;
  }
  int nalloc = 0;
  for (auto &a : allocs) {
    if (a.n == 0 || *a.p != nullptr) continue;  // adopted
    if (++nalloc == fault_alloc)
      return bail(fail(h, LBM_ENOMEM, "injected fault (LBM_FAULT=alloc:K): device allocation refused"));
    cudaError_t e = cudaMalloc(a.p, a.n);
    if (e != cudaSuccess) return bail(cuda_fail(h, e, "cudaMalloc"));
  }
  cudaError_t e = cudaSuccess;
  if (h->sched) {
    e = cudaMemsetAsync(h->sched, 0, 2 * sizeof(unsigned), h->stream);
    if (e != cudaSuccess) return bail(cuda_fail(h, e, "cudaMemset"));
  }
  if (h->dims == 3) {
    // opt in to the largest FD tile any handle may launch (the attribute is
    // per kernel, shared by all handles of the process)
    e = fd3d_configure(P.precision, fd3d_smem_bytes(P.precision, 1));
    if (e != cudaSuccess) return bail(cuda_fail(h, e, "FD shared-memory configuration"));
    // bound of the pipelined FD substep's copy waits (as for the 2D collide below)
    if (P.precision != LBM_F64) {
      unsigned long long wait_ns = 500000000ull;
      if (const char *w = std::getenv("HLBM_DEBUG_TMA_WAIT_NS")) wait_ns = std::strtoull(w, nullptr, 10);
      if (fd3p_set_wait_ns(wait_ns) != 0)
        return bail(fail(h, LBM_ECUDA, "FD copy wait bound: cudaMemcpyToSymbol failed"));
    }
  } else {
    e = collide2d_configure(P.precision);
    if (e != cudaSuccess) return bail(cuda_fail(h, e, "collide shared-memory configuration"));
    // bound of the TMA collide's copy waits: 0.5 s unless HLBM_DEBUG_TMA_WAIT_NS
    // shortens it to exercise the give-up path (process-wide, set at each create)
    if (P.precision != LBM_F64) {
      unsigned long long wait_ns = 500000000ull;
      if (const char *w = std::getenv("HLBM_DEBUG_TMA_WAIT_NS")) wait_ns = std::strtoull(w, nullptr, 10);
      if (collide2d_tma_set_wait_ns(wait_ns) != 0)
        return bail(fail(h, LBM_ECUDA, "TMA wait bound: cudaMemcpyToSymbol failed"));
    }
    int rc2 = autotune_2d(h);
    if (rc2) return bail(rc2);
  }
  *out = h;
  return LBM_OK;
}

int lbm_init_fields(lbm_handle *h, const double *n, const double *phi, const double *ux,
                    const double *uy, const double *uz) {
  int rc = check_usable(h, false);
  if (rc) return rc;
  if (!n || !phi || !ux || !uy || (h->dims == 3 && !uz))
    return fail(h, LBM_EINVAL, "lbm_init_fields: NULL input array");
  bool fault_h2d = false;
  injected_fault(&fault_h2d);
  if (fault_h2d) return fail(h, LBM_ECUDA, "injected fault (LBM_FAULT=h2d): host-to-device copy failed");
  const size_t bytes = sizeof(double) * (size_t)h->S;
  const double *src[5] = {n, phi, ux, uy, uz};
  for (int k = 0; k < 2 + h->dims; k++)
    CK(h, cudaMemcpyAsync(h->staging + k * h->S, src[k], bytes, cudaMemcpyHostToDevice, h->stream),
       "host-to-device copy");
  h->cur = 0;
  CK(h, launch_init(h, 0), "init kernel");
  h->t = 0;
  h->inited = true;
  h->r_ref[0] = h->P.Lx / 2.0;
  h->r_ref[1] = h->P.Ly / 2.0;
  h->r_ref[2] = h->dims == 3 ? h->P.Lz / 2.0 : 0.0;
  CK(h, cudaStreamSynchronize(h->stream), "lbm_init_fields");
  return LBM_OK;
}

int lbm_step(lbm_handle *h, long long nsteps) {
  int rc = check_usable(h, true);
  if (rc) return rc;
  if (nsteps < 0) return fail(h, LBM_EINVAL, "nsteps < 0");
  while (nsteps > 0) {
    const int force_on = h->t < h->P.force_steps;
    const long long len = force_on ? std::min(nsteps, h->P.force_steps - h->t) : nsteps;
    rc = run_segment(h, len, force_on);
    if (rc) return rc;
    nsteps -= len;
  }
  return LBM_OK;
}

int lbm_moments(lbm_handle *h, double *n, double *phi, double *ux, double *uy, double *uz) {
  int rc = check_usable(h, true);
  if (rc) return rc;
  rc = queue_moments(h);
  if (rc) return rc;
  const size_t bytes = sizeof(double) * (size_t)h->S;
  double *dst[5] = {n, phi, ux, uy, uz};
  for (int k = 0; k < 2 + h->dims; k++)
    if (dst[k])
      CK(h, cudaMemcpyAsync(dst[k], h->staging + k * h->S, bytes, cudaMemcpyDeviceToHost, h->stream),
         "device-to-host copy");
  CK(h, cudaStreamSynchronize(h->stream), "lbm_moments");
  if (check_device_waits(h)) return h->err;
  return LBM_OK;
}

int lbm_populations(lbm_handle *h, double *f) {
  int rc = check_usable(h, true);
  if (rc) return rc;
  if (!f) return fail(h, LBM_EINVAL, "lbm_populations: NULL output");
  const size_t bytes = sizeof(double) * (size_t)h->S;
  for (int i = 0; i < h->q; i++) {
    CK(h, launch_population(h, h->cur, i), "population kernel");
    CK(h, cudaMemcpyAsync(f + (size_t)i * h->S, h->staging, bytes, cudaMemcpyDeviceToHost, h->stream),
       "device-to-host copy");
  }
  CK(h, cudaStreamSynchronize(h->stream), "lbm_populations");
  return LBM_OK;
}

int lbm_diagnostics(lbm_handle *h, lbm_diag *out) {
  int rc = check_usable(h, true);
  if (rc) return rc;
  if (!out) return fail(h, LBM_EINVAL, "lbm_diagnostics: NULL output");
  rc = queue_moments(h);
  if (rc) return rc;
  CK(h, launch_diag(h, h->r_ref), "diagnostics kernels");
  double res[DIAG_COUNT];
  CK(h, cudaMemcpyAsync(res, h->dres, sizeof res, cudaMemcpyDeviceToHost, h->stream),
     "device-to-host copy");
  CK(h, cudaStreamSynchronize(h->stream), "lbm_diagnostics");
  if (check_device_waits(h)) return h->err;
  std::memset(out, 0, sizeof *out);
  out->t = h->t;
  out->sum_n = res[DIAG_SUM_N];
  out->sum_phi = res[DIAG_SUM_PHI];
  out->u_max = res[DIAG_UMAX];
  out->dp = res[DIAG_DP];
  out->area = res[DIAG_AREA];
  out->R_eff = h->dims == 2 ? std::sqrt(out->area / M_PI)
                            : std::cbrt(3.0 * out->area / (4.0 * M_PI));
  out->nonfinite = res[DIAG_NONFINITE] != 0.0;
  for (int k = 0; k < h->dims; k++) {
    out->momentum[k] = res[DIAG_MOM0 + k];
    out->r_cm[k] = res[DIAG_RCM0 + k];
    out->v_f[k] = res[DIAG_VF0 + k];
    h->r_ref[k] = out->r_cm[k];
  }
  return out->nonfinite ? LBM_ENONFINITE : LBM_OK;
}

int lbm_synchronize(lbm_handle *h) {
  if (h == nullptr) return LBM_EINVAL;
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) cuda_fail(h, e, "lbm_synchronize");
  check_device_waits(h);
  return h->err;
}

long long lbm_time(const lbm_handle *h) { return h ? h->t : -1; }

int lbm_tuning(const lbm_handle *h, int *values, int n) {
  if (h == nullptr || values == nullptr || n < 0) return LBM_EINVAL;
  const int v[6] = {h->sub, h->fd_rows, h->fd_cols, h->collide_rows, h->m, h->fd_tile_w};
  for (int k = 0; k < n && k < 6; k++) values[k] = v[k];
  return 6;
}
int lbm_fd_substeps(const lbm_handle *h) { return h ? h->m : -1; }

int lbm_set_graphs(lbm_handle *h, int enable) {
  if (h == nullptr) return LBM_EINVAL;
  h->use_graphs = enable != 0;
  return LBM_OK;
}

int lbm_set_kernel_timing(lbm_handle *h, int enable) {
  if (h == nullptr) return LBM_EINVAL;
  h->timing = enable != 0;
  return LBM_OK;
}

int lbm_kernel_times(lbm_handle *h, double *ms, long long *launches, int reset) {
  if (h == nullptr) return LBM_EINVAL;
  harvest_events(h);
  for (int k = 0; k < 3; k++) {
    if (ms) ms[k] = h->ms_acc[k];
    if (launches) launches[k] = h->launches_acc[k];
    if (reset) {
      h->ms_acc[k] = 0;
      h->launches_acc[k] = 0;
    }
  }
  return h->err;
}

int lbm_save(lbm_handle *h, const char *path) {
  int rc = check_usable(h, true);
  if (rc) return rc;
  if (!path) return fail(h, LBM_EINVAL, "lbm_save: NULL path");
  std::vector<unsigned char> buf(h->hbytes + h->phibytes);
  CK(h, cudaMemcpyAsync(buf.data(), h->h[h->cur], h->hbytes, cudaMemcpyDeviceToHost, h->stream),
     "device-to-host copy");
  CK(h, cudaMemcpyAsync(buf.data() + h->hbytes, h->phi[h->cur], h->phibytes,
                        cudaMemcpyDeviceToHost, h->stream),
     "device-to-host copy");
  CK(h, cudaStreamSynchronize(h->stream), "lbm_save");
  CkptHeader hd;
  std::memset(&hd, 0, sizeof hd);
  std::memcpy(hd.magic, "HLBMCKP", 8);
  hd.version = 2;  // 2: lbm_params carries stencil_fd
  hd.t = h->t;
  hd.payload = (long long)buf.size();
  hd.P = h->P;
  hd.crc = crc32_update(0, buf.data(), buf.size());
  FILE *fp = std::fopen(path, "wb");
  if (!fp) return fail(h, LBM_EINVAL, std::string("lbm_save: cannot open ") + path);
  const bool ok = std::fwrite(&hd, sizeof hd, 1, fp) == 1 &&
                  std::fwrite(buf.data(), 1, buf.size(), fp) == buf.size();
  const bool closed = std::fclose(fp) == 0;
  if (!ok || !closed) return fail(h, LBM_EINVAL, std::string("lbm_save: write failed: ") + path);
  return LBM_OK;
}

int lbm_load(lbm_handle *h, const char *path) {
  int rc = check_usable(h, false);
  if (rc) return rc;
  if (!path) return fail(h, LBM_EINVAL, "lbm_load: NULL path");
  FILE *fp = std::fopen(path, "rb");
  if (!fp) return refuse(h, LBM_EINVAL, std::string("lbm_load: cannot open ") + path);
  CkptHeader hd;
  std::vector<unsigned char> buf;
  const char *why = nullptr;
  if (std::fread(&hd, sizeof hd, 1, fp) != 1 || std::memcmp(hd.magic, "HLBMCKP", 8) != 0 ||
      hd.version != 2)
    why = "not a version-2 checkpoint";
  else if (hd.payload != (long long)(h->hbytes + h->phibytes) || !same_params(hd.P, h->P))
    why = "written by a handle with other parameters";
  if (!why) {
    buf.resize(hd.payload);
    if (std::fread(buf.data(), 1, buf.size(), fp) != buf.size()) why = "truncated";
    else if (crc32_update(0, buf.data(), buf.size()) != hd.crc) why = "CRC mismatch";
  }
  std::fclose(fp);
  // a bad file does not poison the handle
  if (why) return refuse(h, LBM_EINVAL, std::string("lbm_load: ") + path + ": " + why);
  CK(h, cudaMemcpyAsync(h->h[0], buf.data(), h->hbytes, cudaMemcpyHostToDevice, h->stream),
     "host-to-device copy");
  CK(h, cudaMemcpyAsync(h->phi[0], buf.data() + h->hbytes, h->phibytes, cudaMemcpyHostToDevice,
                        h->stream),
     "host-to-device copy");
  CK(h, cudaStreamSynchronize(h->stream), "lbm_load");
  h->cur = 0;
  h->t = hd.t;
  h->inited = true;
  return LBM_OK;
}

void lbm_free(lbm_handle *h) {
  if (h == nullptr) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  for (auto &ev : h->events) {
    cudaEventDestroy(ev.a);
    cudaEventDestroy(ev.b);
  }
  for (auto &g : h->graphs) cudaGraphExecDestroy(g.exec);
  void *owned[] = {h->dn, h->staging, h->partials, h->dres, h->fd_a, h->fd_p, h->sched};
  void *lent[] = {h->h[0], h->h[1], h->phi[0], h->phi[1], h->phi[2], h->u};
  for (void *p : owned)
    if (p) cudaFree(p);
  if (!h->adopted)
    for (void *p : lent)
      if (p) cudaFree(p);
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
  delete h;
}

const char *lbm_last_error(const lbm_handle *h) {
  if (h == nullptr) return g_create_error.c_str();
  return h->msg.c_str();
}

}  // extern "C"
