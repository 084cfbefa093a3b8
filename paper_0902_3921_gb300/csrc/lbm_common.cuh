// lbm_common.cuh -- internal declarations shared by the translation units of
// the sm_103a hybrid lattice Boltzmann library: lattice constants, storage
// conversions, kernel parameter blocks, the handle and the kernel launchers.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/hybrid_lbm.h"

namespace hlbm {

// Programmatic dependent launch: a kernel launched with launch_pdl() may be
// scheduled while the previous kernel of the stream is still finishing; it
// calls pdl_wait() before touching anything that kernel wrote (the wait
// returns once that grid has completed and its writes are visible; without
// the launch attribute it returns at once), and pdl_trigger() to let the
// next kernel be scheduled early in turn.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;"); }

bool pdl_enabled();  // HLBM_PDL=1 turns it on (read once; off by default)

// launch_pdl, or a plain launch when pdl is false (the kernel's PDL calls are
// then no-ops)
template <typename... KArgs, typename... Args>
cudaError_t launch_ex(bool pdl, void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                      cudaStream_t stream, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl && pdl_enabled() ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                       cudaStream_t stream, Args... args) {
  return launch_ex(true, kernel, grid, block, smem, stream, args...);
}


// ---- lattices (Sec. II A, Fig. 1; D3Q19 for 3D) --------------------------------
// D2Q9 order: 0 rest; 1..4 = (1,0),(0,1),(-1,0),(0,-1); 5..8 = (1,1),(-1,1),(-1,-1),(1,-1).
__host__ __device__ constexpr int q9_ex(int i) {
  return (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0);
}
__host__ __device__ constexpr int q9_ey(int i) {
  return (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0);
}
__host__ __device__ constexpr double q9_w(int i) {
  return i == 0 ? 4.0 / 9.0 : (i <= 4 ? 1.0 / 9.0 : 1.0 / 36.0);
}
// D3Q19 order: 0 rest; 1..6 faces (+x,-x,+y,-y,+z,-z); 7..18 edges
// (1,1,0),(-1,-1,0),(1,-1,0),(-1,1,0),(1,0,1),(-1,0,-1),(1,0,-1),(-1,0,1),
// (0,1,1),(0,-1,-1),(0,1,-1),(0,-1,1).
__host__ __device__ constexpr int q19_ex(int i) {
  return (i == 1 || i == 7 || i == 9 || i == 11 || i == 13)
             ? 1
             : ((i == 2 || i == 8 || i == 10 || i == 12 || i == 14) ? -1 : 0);
}
__host__ __device__ constexpr int q19_ey(int i) {
  return (i == 3 || i == 7 || i == 10 || i == 15 || i == 17)
             ? 1
             : ((i == 4 || i == 8 || i == 9 || i == 16 || i == 18) ? -1 : 0);
}
__host__ __device__ constexpr int q19_ez(int i) {
  return (i == 5 || i == 11 || i == 14 || i == 15 || i == 18)
             ? 1
             : ((i == 6 || i == 12 || i == 13 || i == 16 || i == 17) ? -1 : 0);
}
__host__ __device__ constexpr double q19_w(int i) {
  return i == 0 ? 1.0 / 3.0 : (i <= 6 ? 1.0 / 18.0 : 1.0 / 36.0);
}

// ---- population storage ----------------------------------------------------------
// Stored value = (f_i - w_i) * scale; scale is 1 except for FP16 storage.
template <typename S, typename C>
struct Store;
template <>
struct Store<double, double> {
  static __device__ __forceinline__ double ld(const double *p, double) { return __ldg(p); }
  static __device__ __forceinline__ void st(double *p, double v, double) { *p = v; }
};
template <>
struct Store<float, float> {
  static __device__ __forceinline__ float ld(const float *p, float) { return __ldg(p); }
  static __device__ __forceinline__ void st(float *p, float v, float) { *p = v; }
};
template <>
struct Store<__half, float> {
  static __device__ __forceinline__ float ld(const __half *p, float inv_scale) {
    return __half2float(__ldg(p)) * inv_scale;
  }
  static __device__ __forceinline__ void st(__half *p, float v, float scale) {
    *p = __float2half_rn(v * scale);
  }
};

// Explicitly rounded operations: code that evaluates one formula in more than
// one place uses them so that every site gets bit-identical results whatever
// contraction the compiler chooses elsewhere.
__device__ __forceinline__ float rn_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double rn_mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float rn_fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double rn_fma(double a, double b, double c) { return __fma_rn(a, b, c); }

__device__ __forceinline__ int wrapi(int x, int L) {
  x %= L;
  return x < 0 ? x + L : x;
}
// Wraps x in [-L, 2L) into [0, L).
__device__ __forceinline__ int wrap1(int x, int L) { return x < 0 ? x + L : (x >= L ? x - L : x); }

// ---- shared-memory addresses and bounded mbarrier waits (bulk-copy pipelines) ----
__device__ __forceinline__ uint32_t su32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Waits for the mbarrier phase `parity` to complete; gives up after limit_ns
// (at once, without polling, when limit_ns is 0: try_wait itself may block
// for a while, long enough for the copies to land).
__device__ __forceinline__ bool bar_wait(uint32_t bar, uint32_t parity, uint64_t limit_ns) {
  if (limit_ns == 0) return false;
  const uint64_t t0 = gtimer();
  while (true) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    if (gtimer() - t0 > limit_ns) return false;
  }
}

// ---- kernel parameter block (host computes it in FP64, kernels read type C) -------
template <typename C>
struct KParams {
  int Lx, Ly, Lz;
  C a, b, kappa;
  C tau_inv, pref;          // 1/tau and 1 - 1/(2 tau) (Eq. 29)
  C N, M, Q, R, C0;         // stencils (Eqs. 30-31); C0 = centre of lap_D
  C gx, gy, gz;             // body force per unit density, 0 when off
  C cs2mT;                  // cs^2 - T (Eq. 28), 0 on the fast path
  C dt, dtG;                // FD step 1/m and Gamma/m (Sec. II C)
  C scale, inv_scale;       // FP16 storage scale 2^s and its inverse (1 otherwise)
  int adv_variant, cubic_at_half;
  int stencil_fd;           // 2D FD: stencil d u (Eq. 30) and lap_D (Eq. 31)
};

// ---- handle -------------------------------------------------------------------
struct GraphEntry {
  long long nsteps;
  int parity;
  int force_on;
  cudaGraphExec_t exec;
};

struct EventPair {
  cudaEvent_t a, b;
  int family;
};

}  // namespace hlbm

struct lbm_handle {
  lbm_params P;
  int dims = 2, q = 9, m = 1, sub = 1;  // sub = FD substeps fused per launch
  int fd_rows = 32;                     // output rows per warp of the 2D FD kernel
  int fd_cols = 4;                      // columns per lane of the 2D FD kernel (FP32)
  int fd_tile_w = 0;                    // 0: marching FD kernel; 32/64: tile kernel width; 128: block; 1: wavefront
  int collide_rows = 2;                 // sites per thread of the 2D collide kernel
  long long S = 0, t = 0;
  bool inited = false;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int cur = 0;  // which of the two population/phi buffers holds time t
  void *h[2] = {nullptr, nullptr};
  void *phi[3] = {nullptr, nullptr, nullptr};  // [2] = FD scratch between launches
  void *fd_a = nullptr, *fd_p = nullptr;        // 3D FP32 FD: phih and psi planes
  bool adopted = false;                        // h, phi, u belong to the caller
  // TMA descriptors of the FP32 collide kernels (CUtensorMap, 128 bytes each):
  // per buffer parity, populations in 32- and 36-column boxes and phi, for
  // 32 x 32 and 32 x 16 tiles
  alignas(64) unsigned char tma_maps[12 * 128] = {};
  bool tma_ready = false;
  unsigned *sched = nullptr;  // tile counter and finished-CTA count of the pipelined collide (2D FP32)
  void *u = nullptr;
  void *dn = nullptr;
  double *staging = nullptr;   // (dims + 3) * S doubles
  double *partials = nullptr;  // diagnostics block partials
  double *dres = nullptr;      // diagnostics result
  double r_ref[3] = {0, 0, 0};
  double phi0 = 1.0;
  size_t hbytes = 0, phibytes = 0;
  int err = 0;
  std::string msg;
  bool use_graphs = true;
  std::vector<hlbm::GraphEntry> graphs;
  bool timing = false;
  std::vector<hlbm::EventPair> events;
  double ms_acc[3] = {0, 0, 0};
  long long launches_acc[3] = {0, 0, 0};
};

namespace hlbm {

// Launchers (return cudaError_t of the launch).  `in`/`out` index the
// population and phi double buffers; force_on selects the body force.
// collide: h[in], phi[in] -> h[1-in], u (STEP) or n, phi, u* as FP64 in staging (MOMENTS)
cudaError_t launch_collide(lbm_handle *h, int in, int force_on, int mode);
// FD update (Sec. II C): phi[in], u -> phi[1-in] (phi[2] between launches)
cudaError_t launch_fd(lbm_handle *h, int in);
// density n - 1 of h[in] into h->dn (only needed when T != 1/3)
cudaError_t launch_density(lbm_handle *h, int in);
// initial state from staging (n, phi, u as FP64) into h[out], phi[out]
cudaError_t launch_init(lbm_handle *h, int out);
// f_i(r, t) of direction i from h[in] into staging[0 .. S) as FP64
cudaError_t launch_population(lbm_handle *h, int in, int i);
// FP64 diagnostics from the MOMENTS staging into h->dres (DIAG_* layout)
cudaError_t launch_diag(lbm_handle *h, const double *r_ref);

// layout of the diagnostics result vector
enum {
  DIAG_SUM_N = 0, DIAG_SUM_PHI, DIAG_MOM0, DIAG_MOM1, DIAG_MOM2, DIAG_UMAX, DIAG_AREA,
  DIAG_CMW, DIAG_CM0, DIAG_CM1, DIAG_CM2, DIAG_NONFINITE, DIAG_NPART,
  // written by the finishing kernel after the partial sums
  DIAG_DP = DIAG_NPART, DIAG_RCM0, DIAG_RCM1, DIAG_RCM2, DIAG_VF0, DIAG_VF1, DIAG_VF2,
  DIAG_COUNT
};
constexpr int DIAG_BLOCKS = 1024;

// mode of launch_collide
enum { COLLIDE_STEP = 0, COLLIDE_MOMENTS = 1 };

template <typename C>
KParams<C> make_params(const lbm_handle *h, int force_on);

// collide with TMA staging (collide2d_tma.cu): FP32 or FP16 deviations,
// Lx % 4 == 0 (FP16: % 8), Lx, Ly >= 64; variant 3: scalar collision, 5 / 6:
// packed pairs budgeted for 4 / 3 CTAs per SM, 7: persistent and pipelined
// (FP32; step mode; the moments mode is always the scalar kernel)
bool collide2d_tma_eligible(const lbm_handle *h, int variant);
cudaError_t collide2d_tma(lbm_handle *h, int in, int force_on, int mode, int variant);
cudaError_t collide2d_tma_configure(int precision);

// FP32 FD update in y-marching form (fd2d_wave.cu): sub = 2 or 4 substeps per
// launch, NY output rows per segment; FP32 or FP16 storage (phi and u* are
// FP32), printed advection form, Lx % 4 == 0, 16-byte aligned phi and u*
bool fd2d_wave_eligible(const lbm_handle *h);
cudaError_t fd2d_wave(lbm_handle *h, const KParams<float> &p, const float *src, float *dst, int sub,
                      int NY);
cudaError_t fd2d_wave_configure();
int fd2d_wave_slots(int sub, int *strips, int Lx);  // CTAs of one wave; strips of Lx
// Batches of independent 2D lattices advanced tile by tile (the tiled path
// of batch.cu): the instance table, the collide over 32 x 16 tiles (items
// (instance, x0, y0, _)) by the tile kernel (kernels_2d.cu) or the pipelined
// TMA kernel (collide2d_tma.cu), and the two-substep wavefront FD over
// 128-column strips (fd2d_wave.cu, items (instance, strip, first output row,
// output rows)).
struct TiledInst {
  int Lx, Ly;
  long long off;  // first site of the instance in the packed planes
  float gx, gy;   // body force per unit density while t < force_steps
  long long force_steps;
};
constexpr int BATCH_TILE_ROWS = 16;
cudaError_t collide2d_batch(const float *hin, float *hout, const float *phi, float *u, long long ST,
                            const TiledInst *inst, const int4 *items, int nitems, const KParams<float> &p,
                            long long t, cudaStream_t s);
int fd2d_wave_batch_strip_columns();  // output columns of a strip
cudaError_t fd2d_wave_batch(const float *phi_in, const float *u, float *phi_out, long long ST,
                            const TiledInst *inst, const int4 *items, int nitems, const KParams<float> &p,
                            cudaStream_t s, bool pdl);
// The TMA collide takes instances at least collide2d_tma_batch_min_side() on
// a side.  The instances of one shape (Lx, Ly) are stored n apart by Lx Ly
// sites from off0 on, so that one set of three tensor maps covers them all
// (populations as an Lx x Ly x n x 9 tensor, phi as Lx x Ly x n); a launch
// takes the maps of up to TMA_BATCH_SHAPES shapes as a kernel parameter, and
// its items carry (shape slot << 16 | index within the shape) in w.
constexpr int TMA_BATCH_SHAPES = 24;
struct TmaShapeMaps {
  alignas(64) unsigned char map[TMA_BATCH_SHAPES][3][128];  // CUtensorMap: p32, p36, phi
  int Lx[TMA_BATCH_SHAPES], Ly[TMA_BATCH_SHAPES];
  long long off0[TMA_BATCH_SHAPES];
};
int collide2d_tma_batch_min_side();
// fills slot `slot` of `m` for the planes h, phi of one buffer parity (false
// if the driver's encoder is missing or refuses the shape)
bool collide2d_tma_batch_shape(TmaShapeMaps *m, int slot, float *h, float *phi, long long ST, int Lx, int Ly,
                               long long off0, int n);
cudaError_t collide2d_tma_batch(const TmaShapeMaps &maps, const float *hin, float *hout, const float *phi,
                                float *u, long long ST, const TiledInst *inst, const int4 *items, int nitems,
                                const KParams<float> &p, long long t, cudaStream_t s, bool pdl);

int collide2d_tma_error(bool reset);  // 1 if a bounded wait of the kernel gave up, -1 on error
int collide2d_tma_set_wait_ns(unsigned long long ns);  // bound of the copy waits (0 on success)
int fd3p_error(bool reset);  // the same for the pipelined 3D FD substep kernel
int fd3p_set_wait_ns(unsigned long long ns);

}  // namespace hlbm
