// kernels_3d.cu -- D3Q19 hot path on sm_103a (the 3D generalisation of the
// paper's D2Q9 scheme).  Same structure as the 2D kernels:
//   collide3d : phi tile + halo 2 in shared memory -> mu (Eq. 5, 19-point lap_D)
//               -> F (Eq. 28, 19-point d_D) -> pull streaming -> n, u* -> BGK
//               with the Guo forcing term (Eqs. 15, 17, 29).
//   fd3d      : `sub` substeps of Eqs. 32-36 (7-point Laplacian) per launch,
//               blocked in shared memory with halo 3 per substep.
//   density3d : n - 1 for the T != 1/3 force term.
// Stencils (3D reading of Eqs. 30-31): d_D has N on the two face neighbours
// along the axis and M on the eight edge neighbours with a non-zero component
// along it (2N + 8M = 1); lap_D has Q on the six faces, R on the twelve edges
// and -(6Q + 12R) at the centre (Q + 4R = 1).
#include <algorithm>
#include <cstdlib>

#include "lbm_common.cuh"

namespace hlbm {

namespace {

constexpr int C3_TX = 32, C3_TY = 8;  // block 32 x 8; z-planes per thread: c3_tz<C>()
template <typename C>
constexpr int c3_tz() {
  return sizeof(C) == 8 ? 4 : 8;  // FP64: the phi and mu tiles must fit 48 KB of static shared memory
}

// Wraps x in [-L, 2L) into [0, L).
__device__ __forceinline__ int wrap1_3(int x, int L) { return x < 0 ? x + L : (x >= L ? x - L : x); }

template <typename S, typename C, bool TGEN, int MODE, int MINB>
__global__ void __launch_bounds__(256, MINB)
    collide3d_kernel(const S *__restrict__ hin, S *__restrict__ hout, const C *__restrict__ phi,
                     const C *__restrict__ dn, C *__restrict__ uout, double *__restrict__ stg,
                     KParams<C> p) {
  constexpr int C3_TZ = c3_tz<C>();
  constexpr int PX = C3_TX + 4, PY = C3_TY + 4, PZ = C3_TZ + 4;
  constexpr int MX = C3_TX + 2, MY = C3_TY + 2, MZ = C3_TZ + 2;
  __shared__ C sphi[PZ][PY][PX];
  __shared__ C smu[MZ][MY][MX];
  const int Lx = p.Lx, Ly = p.Ly, Lz = p.Lz;
  const long long Sz = (long long)Lx * Ly * Lz;
  const int x0 = blockIdx.x * C3_TX, y0 = blockIdx.y * C3_TY, z0 = blockIdx.z * C3_TZ;
  const int tid = threadIdx.y * 32 + threadIdx.x;
  const int lx = threadIdx.x, ly = threadIdx.y, x = x0 + lx, y = y0 + ly;
  const bool site_ok = x < Lx && y < Ly;
  const int xc = site_ok ? x : 0, yc_ = site_ok ? y : 0;
  const int xm = xc == 0 ? Lx - 1 : xc - 1, xp = xc == Lx - 1 ? 0 : xc + 1;
  const int ym = yc_ == 0 ? Ly - 1 : yc_ - 1, yp = yc_ == Ly - 1 ? 0 : yc_ + 1;
  const long long pl = (long long)Lx * Ly;
  const long long yc = (long long)yc_ * Lx, ymo = (long long)ym * Lx, ypo = (long long)yp * Lx;
  // f_i(r) = buf_i(r - e_i) of plane z (clamped into the lattice for threads
  // without a site; their values are never used)
  // FP16 storage: the populations stay in their stored scale 2^s through the
  // sums and the collision (the scale is folded into the moments and the
  // weights), which is exact for a power of two and saves a multiply per
  // population read and written
  constexpr bool FOLD = !std::is_same<S, C>::value;
  const C ld_scale = FOLD ? C(1) : p.inv_scale, st_scale = FOLD ? C(1) : p.scale;
  const C wsc = FOLD ? p.scale : C(1);  // weights in the stored scale
  auto load_plane = [&](C (&hv)[19], int z) {
    const int zm = z == 0 ? Lz - 1 : z - 1, zp = z == Lz - 1 ? 0 : z + 1;
    const long long zc = (long long)z * pl, zmo = (long long)zm * pl, zpo = (long long)zp * pl;
#define LD(i, zz, yy, xx) hv[i] = Store<S, C>::ld(hin + (i)*Sz + (zz) + (yy) + (xx), ld_scale)
    LD(0, zc, yc, xc);
    LD(1, zc, yc, xm);
    LD(2, zc, yc, xp);
    LD(3, zc, ymo, xc);
    LD(4, zc, ypo, xc);
    LD(5, zmo, yc, xc);
    LD(6, zpo, yc, xc);
    LD(7, zc, ymo, xm);    // (1,1,0)
    LD(8, zc, ypo, xp);    // (-1,-1,0)
    LD(9, zc, ypo, xm);    // (1,-1,0)
    LD(10, zc, ymo, xp);   // (-1,1,0)
    LD(11, zmo, yc, xm);   // (1,0,1)
    LD(12, zpo, yc, xp);   // (-1,0,-1)
    LD(13, zpo, yc, xm);   // (1,0,-1)
    LD(14, zmo, yc, xp);   // (-1,0,1)
    LD(15, zmo, ymo, xc);  // (0,1,1)
    LD(16, zpo, ypo, xc);  // (0,-1,-1)
    LD(17, zpo, ymo, xc);  // (0,1,-1)
    LD(18, zmo, ypo, xc);  // (0,-1,1)
#undef LD
  };
  // the first plane's populations are in flight while phi and mu are staged
  C hv[19], hn[19];
  if (z0 < Lz) load_plane(hv, z0);
  const bool big = Lx >= PX && Ly >= PY && Lz >= PZ;
  // phi on the tile + halo 2: one (x, y) column per thread, the z loop inside
  for (int k = tid; k < PX * PY; k += 256) {
    const int ry = k / PX, rx = k - ry * PX;
    const int gx = big ? wrap1_3(x0 + rx - 2, Lx) : wrapi(x0 + rx - 2, Lx);
    const int gy = big ? wrap1_3(y0 + ry - 2, Ly) : wrapi(y0 + ry - 2, Ly);
    const C *col = phi + (long long)gy * Lx + gx;
    C v[PZ];  // the whole column in flight before any of it is stored
#pragma unroll
    for (int rz = 0; rz < PZ; ++rz) {
      const int gz = big ? wrap1_3(z0 + rz - 2, Lz) : wrapi(z0 + rz - 2, Lz);
      v[rz] = col[(long long)gz * pl];
    }
#pragma unroll
    for (int rz = 0; rz < PZ; ++rz) sphi[rz][ry][rx] = v[rz];
  }
  __syncthreads();
  // mu on the tile + 1: one (x, y) column per thread marching in z, the 3 x 3
  // neighbourhoods of phi on planes z - 1, z, z + 1 in registers (9 new
  // loads per site)
  for (int k = tid; k < MX * MY; k += 256) {
    const int my = k / MX, mx = k - my * MX, cy = my + 1, cx = mx + 1;
    C w[3][3][3];  // [plane][dy][dx]
#pragma unroll
    for (int pz = 0; pz < 2; ++pz)
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) w[pz + 1][a][b] = sphi[pz][cy - 1 + a][cx - 1 + b];
#pragma unroll 2
    for (int mz = 0; mz < MZ; ++mz) {
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
          w[0][a][b] = w[1][a][b];
          w[1][a][b] = w[2][a][b];
          w[2][a][b] = sphi[mz + 2][cy - 1 + a][cx - 1 + b];
        }
      const C c = w[1][1][1];
      const C faces = ((w[1][1][0] + w[1][1][2]) + (w[1][0][1] + w[1][2][1])) + (w[0][1][1] + w[2][1][1]);
      const C edges = ((w[1][0][0] + w[1][0][2]) + (w[1][2][0] + w[1][2][2])) +
                      ((w[0][1][0] + w[0][1][2]) + (w[2][1][0] + w[2][1][2])) +
                      ((w[0][0][1] + w[0][2][1]) + (w[2][0][1] + w[2][2][1]));
      const C lap = p.Q * faces + p.R * edges + p.C0 * c;
      smu[mz][my][mx] = p.a * c + p.b * c * c * c - p.kappa * lap;
    }
  }
  __syncthreads();

  if (!site_ok) return;
#pragma unroll 1
  for (int lz = 0; lz < C3_TZ; ++lz) {
    const int z = z0 + lz;
    if (z >= Lz) break;
    // the next plane's populations are issued before this plane is computed
    if (lz + 1 < C3_TZ && z + 1 < Lz) load_plane(hn, z + 1);
    const int mx = lx + 1, my = ly + 1, mz = lz + 1;
    // d_D mu along x, y, z
    auto grad = [&](const C (*f)[MY][MX], C &gx_, C &gy_, C &gz_) {
      gx_ = p.N * (f[mz][my][mx + 1] - f[mz][my][mx - 1]) +
            p.M * (((f[mz][my - 1][mx + 1] - f[mz][my - 1][mx - 1]) +
                    (f[mz][my + 1][mx + 1] - f[mz][my + 1][mx - 1])) +
                   ((f[mz - 1][my][mx + 1] - f[mz - 1][my][mx - 1]) +
                    (f[mz + 1][my][mx + 1] - f[mz + 1][my][mx - 1])));
      gy_ = p.N * (f[mz][my + 1][mx] - f[mz][my - 1][mx]) +
            p.M * (((f[mz][my + 1][mx - 1] - f[mz][my - 1][mx - 1]) +
                    (f[mz][my + 1][mx + 1] - f[mz][my - 1][mx + 1])) +
                   ((f[mz - 1][my + 1][mx] - f[mz - 1][my - 1][mx]) +
                    (f[mz + 1][my + 1][mx] - f[mz + 1][my - 1][mx])));
      gz_ = p.N * (f[mz + 1][my][mx] - f[mz - 1][my][mx]) +
            p.M * (((f[mz + 1][my][mx - 1] - f[mz - 1][my][mx - 1]) +
                    (f[mz + 1][my][mx + 1] - f[mz - 1][my][mx + 1])) +
                   ((f[mz + 1][my - 1][mx] - f[mz - 1][my - 1][mx]) +
                    (f[mz + 1][my + 1][mx] - f[mz - 1][my + 1][mx])));
    };
    C gmx, gmy, gmz;
    grad(smu, gmx, gmy, gmz);
    const C ph = sphi[lz + 2][ly + 2][lx + 2];
    C Fx = -ph * gmx, Fy = -ph * gmy, Fz = -ph * gmz;
    if constexpr (TGEN) {
      // d_D((cs2 - T) n) from the density pass, read directly (rare path)
      auto pn = [&](int dx, int dy, int dz) {
        const long long g = ((long long)wrapi(z + dz, Lz) * Ly + wrapi(y + dy, Ly)) * Lx +
                            wrapi(x + dx, Lx);
        return p.cs2mT * (C(1) + dn[g]);
      };
      Fx += p.N * (pn(1, 0, 0) - pn(-1, 0, 0)) +
            p.M * (((pn(1, -1, 0) - pn(-1, -1, 0)) + (pn(1, 1, 0) - pn(-1, 1, 0))) +
                   ((pn(1, 0, -1) - pn(-1, 0, -1)) + (pn(1, 0, 1) - pn(-1, 0, 1))));
      Fy += p.N * (pn(0, 1, 0) - pn(0, -1, 0)) +
            p.M * (((pn(-1, 1, 0) - pn(-1, -1, 0)) + (pn(1, 1, 0) - pn(1, -1, 0))) +
                   ((pn(0, 1, -1) - pn(0, -1, -1)) + (pn(0, 1, 1) - pn(0, -1, 1))));
      Fz += p.N * (pn(0, 0, 1) - pn(0, 0, -1)) +
            p.M * (((pn(-1, 0, 1) - pn(-1, 0, -1)) + (pn(1, 0, 1) - pn(1, 0, -1))) +
                   ((pn(0, -1, 1) - pn(0, -1, -1)) + (pn(0, 1, 1) - pn(0, 1, -1))));
    }
    const long long zc = (long long)z * pl;
    C dens = hv[0];
#pragma unroll
    for (int i = 1; i < 19; ++i) dens += hv[i];
    C jx = C(0), jy = C(0), jz = C(0);
#pragma unroll
    for (int i = 1; i < 19; ++i) {
      if (q19_ex(i) > 0) jx += hv[i];
      if (q19_ex(i) < 0) jx -= hv[i];
      if (q19_ey(i) > 0) jy += hv[i];
      if (q19_ey(i) < 0) jy -= hv[i];
      if (q19_ez(i) > 0) jz += hv[i];
      if (q19_ez(i) < 0) jz -= hv[i];
    }
    if constexpr (FOLD) {
      dens *= p.inv_scale;
      jx *= p.inv_scale;
      jy *= p.inv_scale;
      jz *= p.inv_scale;
    }
    const C n = C(1) + dens;
    Fx += n * p.gx;
    Fy += n * p.gy;
    Fz += n * p.gz;
    const C inv_n = C(1) / n;
    const C ux = (jx + C(0.5) * Fx) * inv_n;
    const C uy = (jy + C(0.5) * Fy) * inv_n;
    const C uz = (jz + C(0.5) * Fz) * inv_n;
    const long long s = zc + yc + x;
    if constexpr (MODE == COLLIDE_MOMENTS) {
      stg[s] = (double)n;
      stg[Sz + s] = (double)ph;
      stg[2 * Sz + s] = (double)ux;
      stg[3 * Sz + s] = (double)uy;
      stg[4 * Sz + s] = (double)uz;
#pragma unroll
      for (int i = 0; i < 19; ++i) hv[i] = hn[i];
      continue;
    }
    const C usq = ux * ux + uy * uy + uz * uz;
    const C uF = ux * Fx + uy * Fy + uz * Fz;
    const C om = p.tau_inv, keep = C(1) - p.tau_inv;
    const C base = dens - n * (C(1.5) * usq);  // the u-independent and |u|^2 parts
    if constexpr (FOLD) {
      // BGK + Guo source (Eqs. 15, 17, 29) per opposite pair (i, i + 1): with
      // A = w / tau and B = w (1 - 1/2tau) per weight class, the part even in
      // e_i is E = A (base + 4.5 n (e.u)^2) + B (9 (e.u)(e.F) - 3 u.F) and the
      // odd part O = 3 A n (e.u) + 3 B (e.F); f_i = (1 - 1/tau) f_i + E + O,
      // f_ib = (1 - 1/tau) f_ib + E - O.  e.u and e.F take only the non-zero
      // components of e_i (the compiler may not drop a product with a zero
      // component under IEEE rules).  FP16 storage only: the kernel is
      // issue-bound there (417 against 444 us a launch at 256^3), while the
      // FP32 kernel, closer to the memory roof, ran slower with this form
      // (473 against 464 us), so it keeps the one below.
      const C n45 = C(4.5) * n, m3uF = C(-3) * uF;
      const C A0 = om * C(q19_w(0)) * wsc, B0 = p.pref * C(q19_w(0)) * wsc;
      const C A1 = om * C(q19_w(1)) * wsc, B1 = p.pref * C(q19_w(1)) * wsc;  // faces
      const C A2 = om * C(q19_w(7)) * wsc, B2 = p.pref * C(q19_w(7)) * wsc;  // edges
      const C An3_1 = C(3) * A1 * n, An3_2 = C(3) * A2 * n;
      Store<S, C>::st(hout + s, keep * hv[0] + (A0 * base + B0 * m3uF), st_scale);
      auto edot = [](int ex, int ey, int ez, C a, C b, C c) {
        C r = ex > 0 ? a : (ex < 0 ? -a : C(0));
        if (ey != 0) r = ex != 0 ? (ey > 0 ? r + b : r - b) : (ey > 0 ? b : -b);
        if (ez != 0) r = (ex != 0 || ey != 0) ? (ez > 0 ? r + c : r - c) : (ez > 0 ? c : -c);
        return r;
      };
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        const int i = 2 * k + 1, ib = i + 1;  // e_ib = -e_i
        const bool face = k < 3;
        const C A = face ? A1 : A2, B = face ? B1 : B2, An3 = face ? An3_1 : An3_2;
        const C eu = edot(q19_ex(i), q19_ey(i), q19_ez(i), ux, uy, uz);
        const C eF = edot(q19_ex(i), q19_ey(i), q19_ez(i), Fx, Fy, Fz);
        const C se = n45 * eu * eu + base;
        const C fe = C(9) * eu * eF + m3uF;
        const C E = A * se + B * fe;
        const C O = An3 * eu + C(3) * B * eF;
        Store<S, C>::st(hout + i * Sz + s, (keep * hv[i] + E) + O, st_scale);
        Store<S, C>::st(hout + ib * Sz + s, (keep * hv[ib] + E) - O, st_scale);
      }
    } else {
      // BGK + Guo source (Eqs. 15, 17, 29) per opposite pair (i, i + 1): the
      // parts even and odd in e_i are formed once and added / subtracted
      const C n3 = C(3) * n, n45 = C(4.5) * n;
      const C pF3 = C(3) * p.pref, pF9 = C(9) * p.pref, puF = C(3) * p.pref * uF;
      {
        const C w = C(q19_w(0));
        Store<S, C>::st(hout + s, keep * hv[0] + om * (w * base) + w * (-puF), st_scale);
      }
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        const int i = 2 * k + 1, ib = i + 1;  // e_ib = -e_i
        const C w = C(q19_w(i));
        const C eu = C(q19_ex(i)) * ux + C(q19_ey(i)) * uy + C(q19_ez(i)) * uz;
        const C eF = C(q19_ex(i)) * Fx + C(q19_ey(i)) * Fy + C(q19_ez(i)) * Fz;
        const C even = w * (base + n45 * eu * eu);
        const C odd = w * (n3 * eu);
        const C Feven = w * (pF9 * eu * eF - puF);
        const C Fodd = w * (pF3 * eF);
        Store<S, C>::st(hout + i * Sz + s, keep * hv[i] + om * (even + odd) + (Feven + Fodd), st_scale);
        Store<S, C>::st(hout + ib * Sz + s, keep * hv[ib] + om * (even - odd) + (Feven - Fodd), st_scale);
      }
    }
    uout[s] = ux;
    uout[Sz + s] = uy;
    uout[2 * Sz + s] = uz;
#pragma unroll
    for (int i = 0; i < 19; ++i) hv[i] = hn[i];
  }
}

template <typename C, int TX, int TY, int TZ>
__global__ void __launch_bounds__(256)
    fd3d_kernel(const C *__restrict__ phi_in, const C *__restrict__ u, C *__restrict__ phi_out,
                KParams<C> p, int sub) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C *sm = reinterpret_cast<C *>(smem_raw);
  const int H = 3 * sub, RX = TX + 2 * H, RY = TY + 2 * H, RZ = TZ + 2 * H;
  const int R = RX * RY * RZ, PL = RX * RY;
  C *sp = sm, *sh = sm + R, *sq = sm + 2 * R, *su = sm + 3 * R, *sv = sm + 4 * R,
    *sw = sm + 5 * R;
  const int Lx = p.Lx, Ly = p.Ly, Lz = p.Lz;
  const long long Sz = (long long)Lx * Ly * Lz;
  const int x0 = blockIdx.x * TX - H, y0 = blockIdx.y * TY - H, z0 = blockIdx.z * TZ - H;
  const int tx = threadIdx.x, ty = threadIdx.y;
  for (int rz = 0; rz < RZ; ++rz)
    for (int ry = ty; ry < RY; ry += 8) {
      const long long row = ((long long)wrapi(z0 + rz, Lz) * Ly + wrapi(y0 + ry, Ly)) * Lx;
      for (int rx = tx; rx < RX; rx += 32) {
        const long long g = row + wrapi(x0 + rx, Lx);
        const int k = rz * PL + ry * RX + rx;
        sp[k] = phi_in[g];
        su[k] = u[g];
        sv[k] = u[Sz + g];
        sw[k] = u[2 * Sz + g];
      }
    }
  __syncthreads();
  const C dt = p.dt, dtG = p.dtG;
#pragma unroll 1
  for (int s = 1; s <= sub; ++s) {
    int lo = 3 * s - 2;
    for (int rz = lo; rz < RZ - lo; ++rz)
      for (int ry = lo + ty; ry < RY - lo; ry += 8)
        for (int rx = lo + tx; rx < RX - lo; rx += 32) {
          const int k = rz * PL + ry * RX + rx;
          const C ph = sp[k];
          C tend;
          if (p.adv_variant == LBM_ADV_PAPER) {
            const C ua = su[k], va = sv[k], wa = sw[k];
            const C dux = (su[k + 1] - su[k - 1]) / C(2);
            const C dpx = ua < C(0) ? sp[k + 1] - ph : ph - sp[k - 1];
            const C duy = (sv[k + RX] - sv[k - RX]) / C(2);
            const C dpy = va < C(0) ? sp[k + RX] - ph : ph - sp[k - RX];
            const C duz = (sw[k + PL] - sw[k - PL]) / C(2);
            const C dpz = wa < C(0) ? sp[k + PL] - ph : ph - sp[k - PL];
            tend = (ph * dux + ua * dpx);
            tend += (ph * duy + va * dpy);
            tend += (ph * duz + wa * dpz);
          } else {
            auto flux = [&](const C *uu, int st) {
              const C Up = C(0.5) * (uu[k] + uu[k + st]);
              const C Um = C(0.5) * (uu[k - st] + uu[k]);
              const C Jp = Up > C(0) ? Up * ph : Up * sp[k + st];
              const C Jm = Um > C(0) ? Um * sp[k - st] : Um * ph;
              return Jp - Jm;
            };
            tend = flux(su, 1);
            tend += flux(sv, RX);
            tend += flux(sw, PL);
          }
          sh[k] = ph - dt * tend;
        }
    __syncthreads();
    lo = 3 * s - 1;
    for (int rz = lo; rz < RZ - lo; ++rz)
      for (int ry = lo + ty; ry < RY - lo; ry += 8)
        for (int rx = lo + tx; rx < RX - lo; rx += 32) {
          const int k = rz * PL + ry * RX + rx;
          const C hk = sh[k];
          const C c = p.cubic_at_half ? hk : sp[k];
          C lap = sh[k - PL];
          lap += sh[k - RX];
          lap += sh[k - 1];
          lap += C(-6) * hk;
          lap += sh[k + 1];
          lap += sh[k + RX];
          lap += sh[k + PL];
          sq[k] = p.a * hk + p.b * (c * c * c) - p.kappa * lap;
        }
    __syncthreads();
    lo = 3 * s;
    for (int rz = lo; rz < RZ - lo; ++rz)
      for (int ry = lo + ty; ry < RY - lo; ry += 8)
        for (int rx = lo + tx; rx < RX - lo; rx += 32) {
          const int k = rz * PL + ry * RX + rx;
          C lap = sq[k - PL];
          lap += sq[k - RX];
          lap += sq[k - 1];
          lap += C(-6) * sq[k];
          lap += sq[k + 1];
          lap += sq[k + RX];
          lap += sq[k + PL];
          sp[k] = sh[k] + dtG * lap;
        }
    __syncthreads();
  }
  for (int rz = H; rz < H + TZ; ++rz) {
    const int gz = z0 + rz;
    if (gz >= Lz) break;
    for (int ry = H + ty; ry < H + TY; ry += 8) {
      const int gy = y0 + ry;
      if (gy >= Ly) break;
      for (int rx = H + tx; rx < H + TX; rx += 32) {
        const int gx = x0 + rx;
        if (gx < Lx) phi_out[((long long)gz * Ly + gy) * Lx + gx] = sp[rz * PL + ry * RX + rx];
      }
    }
  }
}

// ---- FD 3D, FP32: three passes per substep --------------------------------------
// One site per thread over the whole lattice, periodic neighbours by index
// arithmetic; no halo is recomputed.  Pass 1: phih (Eqs. 32-35) from the
// 7-point neighbourhood of phi and u*; pass 2: psi = a phih + b phi^3 -
// kappa lap phih (Eq. 36); pass 3: phi^{n+1} = phih + dt Gamma lap psi.  The
// expressions are those of fd3d_kernel, in the same order.
struct Nbr3 {
  long long s, xm, xp, ym, yp, zm, zp;
};

__device__ __forceinline__ bool nbr3(const KParams<float> &p, Nbr3 &n) {
  const int Lx = p.Lx, Ly = p.Ly, Lz = p.Lz;
  const int x = blockIdx.x * 32 + threadIdx.x, y = blockIdx.y * 8 + threadIdx.y, z = blockIdx.z;
  if (x >= Lx || y >= Ly) return false;
  const long long PL = (long long)Lx * Ly;
  n.s = z * PL + (long long)y * Lx + x;
  n.xm = n.s + (x == 0 ? Lx - 1 : -1);
  n.xp = n.s + (x == Lx - 1 ? 1 - Lx : 1);
  n.ym = n.s + (y == 0 ? (long long)(Ly - 1) * Lx : -(long long)Lx);
  n.yp = n.s + (y == Ly - 1 ? -(long long)(Ly - 1) * Lx : (long long)Lx);
  n.zm = n.s + (z == 0 ? (Lz - 1) * PL : -PL);
  n.zp = n.s + (z == Lz - 1 ? -(Lz - 1) * PL : PL);
  return true;
}

template <bool FLUX>
__global__ void __launch_bounds__(256)
    fd3_adv_kernel(const float *__restrict__ phi, const float *__restrict__ u,
                   float *__restrict__ A, KParams<float> p) {
  Nbr3 n;
  if (!nbr3(p, n)) return;
  const long long Sz = (long long)p.Lx * p.Ly * p.Lz;
  const float *v = u + Sz, *w = u + 2 * Sz;
  const float ph = __ldg(phi + n.s);
  float tend;
  if constexpr (!FLUX) {
    const float ua = __ldg(u + n.s), va = __ldg(v + n.s), wa = __ldg(w + n.s);
    const float dux = (__ldg(u + n.xp) - __ldg(u + n.xm)) / 2.f;
    const float dpx = ua < 0.f ? __ldg(phi + n.xp) - ph : ph - __ldg(phi + n.xm);
    const float duy = (__ldg(v + n.yp) - __ldg(v + n.ym)) / 2.f;
    const float dpy = va < 0.f ? __ldg(phi + n.yp) - ph : ph - __ldg(phi + n.ym);
    const float duz = (__ldg(w + n.zp) - __ldg(w + n.zm)) / 2.f;
    const float dpz = wa < 0.f ? __ldg(phi + n.zp) - ph : ph - __ldg(phi + n.zm);
    tend = (ph * dux + ua * dpx);
    tend += (ph * duy + va * dpy);
    tend += (ph * duz + wa * dpz);
  } else {
    auto flux = [&](const float *uu, long long m, long long q) {
      const float uc = __ldg(uu + n.s);
      const float Up = 0.5f * (uc + __ldg(uu + q));
      const float Um = 0.5f * (__ldg(uu + m) + uc);
      const float Jp = Up > 0.f ? Up * ph : Up * __ldg(phi + q);
      const float Jm = Um > 0.f ? Um * __ldg(phi + m) : Um * ph;
      return Jp - Jm;
    };
    tend = flux(u, n.xm, n.xp);
    tend += flux(v, n.ym, n.yp);
    tend += flux(w, n.zm, n.zp);
  }
  A[n.s] = ph - p.dt * tend;
}

__global__ void __launch_bounds__(256)
    fd3_psi_kernel(const float *__restrict__ A, const float *__restrict__ phi,
                   float *__restrict__ P, KParams<float> p) {
  Nbr3 n;
  if (!nbr3(p, n)) return;
  const float hk = __ldg(A + n.s);
  const float c = p.cubic_at_half ? hk : __ldg(phi + n.s);
  float lap = __ldg(A + n.zm);
  lap += __ldg(A + n.ym);
  lap += __ldg(A + n.xm);
  lap += -6.f * hk;
  lap += __ldg(A + n.xp);
  lap += __ldg(A + n.yp);
  lap += __ldg(A + n.zp);
  P[n.s] = p.a * hk + p.b * (c * c * c) - p.kappa * lap;
}

__global__ void __launch_bounds__(256)
    fd3_phi_kernel(const float *__restrict__ P, const float *__restrict__ A,
                   float *__restrict__ phi_out, KParams<float> p) {
  Nbr3 n;
  if (!nbr3(p, n)) return;
  float lap = __ldg(P + n.zm);
  lap += __ldg(P + n.ym);
  lap += __ldg(P + n.xm);
  lap += -6.f * __ldg(P + n.s);
  lap += __ldg(P + n.xp);
  lap += __ldg(P + n.yp);
  lap += __ldg(P + n.zp);
  phi_out[n.s] = __ldg(A + n.s) + p.dtG * lap;
}

// ---- the same three passes, four x-sites per thread, marching in z ------------
// (Lx a multiple of 4.)  A warp covers 128 consecutive x (float4 per lane, the
// x neighbours by shuffles; lanes at a warp or lattice edge load their wrapped
// neighbour), a block 8 rows of y, and each thread marches nz planes in z
// (at most F3V_NZ, fewer when the lattice is too small to fill the GPU)
// keeping the z-1, z, z+1 values of the marched field in registers.
constexpr int F3V_NZ = 16;

struct Vq {
  int x4, xc, y, z0, z1, lane;
  bool ok;
};

__device__ __forceinline__ Vq vq_of(const KParams<float> &p, int nz) {
  Vq q;
  q.lane = threadIdx.x;
  q.x4 = 4 * (blockIdx.x * 32 + threadIdx.x);
  q.xc = min(q.x4, p.Lx - 4);  // loads of lanes past the lattice edge stay in bounds
  q.ok = q.x4 < p.Lx;
  q.y = blockIdx.y * 8 + threadIdx.y;
  q.z0 = blockIdx.z * nz;
  q.z1 = min(q.z0 + nz, p.Lz);
  return q;
}

__device__ __forceinline__ const float *row_of(const float *a, int y, int z, const KParams<float> &p) {
  return a + ((long long)z * p.Ly + y) * p.Lx;
}

__device__ __forceinline__ float4 ld4g(const float *row, int x) {
  return __ldg(reinterpret_cast<const float4 *>(row + x));
}

// values at x4 - 1 and x4 + 4 of `row`, whose quad at x4 is c
__device__ __forceinline__ void xnbr4(const float *row, float4 c, const Vq &q, int Lx, float &l,
                                      float &r) {
  l = __shfl_up_sync(0xffffffffu, c.w, 1);
  r = __shfl_down_sync(0xffffffffu, c.x, 1);
  if (q.lane == 0 || q.x4 == 0) l = __ldg(row + (q.x4 == 0 ? Lx - 1 : q.xc - 1));
  if (q.lane == 31 || q.x4 + 4 >= Lx) r = __ldg(row + (q.x4 + 4 >= Lx ? 0 : q.x4 + 4));
}

__device__ __forceinline__ float cmp4(const float4 &v, int j) {
  return j == 0 ? v.x : (j == 1 ? v.y : (j == 2 ? v.z : v.w));
}

// phih of one site (Eqs. 32-35, or the flux form): phi at the site and its
// six neighbours, the u* components along each axis at the neighbours that
// the central divergence (or the face velocities) needs
template <bool FLUX>
__device__ __forceinline__ float adv_site(float ph, float pxm, float pxp, float pym, float pyp, float pzm,
                                          float pzp, float uxm, float ua, float uxp, float vym, float va,
                                          float vyp, float wzm, float wa, float wzp, float dt) {
  float tend;
  if constexpr (!FLUX) {
    const float dux = (uxp - uxm) / 2.f;
    const float dpx = ua < 0.f ? pxp - ph : ph - pxm;
    const float duy = (vyp - vym) / 2.f;
    const float dpy = va < 0.f ? pyp - ph : ph - pym;
    const float duz = (wzp - wzm) / 2.f;
    const float dpz = wa < 0.f ? pzp - ph : ph - pzm;
    tend = (ph * dux + ua * dpx);
    tend += (ph * duy + va * dpy);
    tend += (ph * duz + wa * dpz);
  } else {
    auto flux = [&](float cm, float cc, float cp, float fm, float fp) {
      const float Up = 0.5f * (cc + cp);
      const float Um = 0.5f * (cm + cc);
      const float Jp = Up > 0.f ? Up * ph : Up * fp;
      const float Jm = Um > 0.f ? Um * fm : Um * ph;
      return Jp - Jm;
    };
    tend = flux(uxm, ua, uxp, pxm, pxp);
    tend += flux(vym, va, vyp, pym, pyp);
    tend += flux(wzm, wa, wzp, pzm, pzp);
  }
  return ph - dt * tend;
}

template <bool FLUX>
__global__ void __launch_bounds__(256)
    fd3v_adv_kernel(const float *__restrict__ phi, const float *__restrict__ u,
                    float *__restrict__ A, KParams<float> p, int nz) {
  const Vq q = vq_of(p, nz);
  if (q.y >= p.Ly) return;  // warp-uniform (a warp is one row)
  const int Lx = p.Lx, Ly = p.Ly, Lz = p.Lz;
  const long long Sz = (long long)Lx * Ly * Lz;
  const float *v = u + Sz, *w = u + 2 * Sz;
  const int ym = q.y == 0 ? Ly - 1 : q.y - 1, yp = q.y == Ly - 1 ? 0 : q.y + 1;
  const int zb = q.z0 == 0 ? Lz - 1 : q.z0 - 1;
  float4 pm = ld4g(row_of(phi, q.y, zb, p), q.xc), pc = ld4g(row_of(phi, q.y, q.z0, p), q.xc);
  float4 wm = ld4g(row_of(w, q.y, zb, p), q.xc), wc = ld4g(row_of(w, q.y, q.z0, p), q.xc);
  for (int z = q.z0; z < q.z1; ++z) {
    const int zn = z == Lz - 1 ? 0 : z + 1;
    const float *prow = row_of(phi, q.y, z, p), *urow = row_of(u, q.y, z, p);
    const float4 pp = ld4g(row_of(phi, q.y, zn, p), q.xc), wp = ld4g(row_of(w, q.y, zn, p), q.xc);
    const float4 pym = ld4g(row_of(phi, ym, z, p), q.xc), pyp = ld4g(row_of(phi, yp, z, p), q.xc);
    const float4 uc = ld4g(urow, q.xc), vc = ld4g(row_of(v, q.y, z, p), q.xc);
    const float4 vym = ld4g(row_of(v, ym, z, p), q.xc), vyp = ld4g(row_of(v, yp, z, p), q.xc);
    float pl, pr, ul, ur;
    xnbr4(prow, pc, q, Lx, pl, pr);
    xnbr4(urow, uc, q, Lx, ul, ur);
    float e[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const float ph = cmp4(pc, j);
      const float pxm = j == 0 ? pl : cmp4(pc, j - 1), pxp = j == 3 ? pr : cmp4(pc, j + 1);
      const float uxm = j == 0 ? ul : cmp4(uc, j - 1), uxp = j == 3 ? ur : cmp4(uc, j + 1);
      e[j] = adv_site<FLUX>(ph, pxm, pxp, cmp4(pym, j), cmp4(pyp, j), cmp4(pm, j), cmp4(pp, j), uxm,
                            cmp4(uc, j), uxp, cmp4(vym, j), cmp4(vc, j), cmp4(vyp, j), cmp4(wm, j),
                            cmp4(wc, j), cmp4(wp, j), p.dt);
    }
    if (q.ok)
      *reinterpret_cast<float4 *>(A + ((long long)z * Ly + q.y) * Lx + q.x4) =
          make_float4(e[0], e[1], e[2], e[3]);
    pm = pc;
    pc = pp;
    wm = wc;
    wc = wp;
  }
}

// LAP7 of a field with the quad c at (y, z) and its neighbours, in the order
// z-1, y-1, x-1, centre, x+1, y+1, z+1 of the scalar kernels
template <bool PSI>
__global__ void __launch_bounds__(256)
    fd3v_lap_kernel(const float *__restrict__ F, const float *__restrict__ G,
                    float *__restrict__ out, KParams<float> p, int nz) {
  // PSI:  out = a F + b c^3 - kappa lap F, c = (cubic_at_half ? F : G)
  // else: out = G + dtG lap F
  const Vq q = vq_of(p, nz);
  if (q.y >= p.Ly) return;
  const int Lx = p.Lx, Ly = p.Ly, Lz = p.Lz;
  const int ym = q.y == 0 ? Ly - 1 : q.y - 1, yp = q.y == Ly - 1 ? 0 : q.y + 1;
  const int zb = q.z0 == 0 ? Lz - 1 : q.z0 - 1;
  float4 fm = ld4g(row_of(F, q.y, zb, p), q.xc), fc = ld4g(row_of(F, q.y, q.z0, p), q.xc);
  for (int z = q.z0; z < q.z1; ++z) {
    const int zn = z == Lz - 1 ? 0 : z + 1;
    const float *frow = row_of(F, q.y, z, p);
    const float4 fp = ld4g(row_of(F, q.y, zn, p), q.xc);
    const float4 fym = ld4g(row_of(F, ym, z, p), q.xc), fyp = ld4g(row_of(F, yp, z, p), q.xc);
    const float4 gc = ld4g(row_of(G, q.y, z, p), q.xc);
    float fl, fr;
    xnbr4(frow, fc, q, Lx, fl, fr);
    float e[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const float hk = cmp4(fc, j);
      float lap = cmp4(fm, j);
      lap += cmp4(fym, j);
      lap += j == 0 ? fl : cmp4(fc, j - 1);
      lap += -6.f * hk;
      lap += j == 3 ? fr : cmp4(fc, j + 1);
      lap += cmp4(fyp, j);
      lap += cmp4(fp, j);
      if constexpr (PSI) {
        const float c = p.cubic_at_half ? hk : cmp4(gc, j);
        e[j] = p.a * hk + p.b * (c * c * c) - p.kappa * lap;
      } else {
        e[j] = cmp4(gc, j) + p.dtG * lap;
      }
    }
    if (q.ok)
      *reinterpret_cast<float4 *>(out + ((long long)z * Ly + q.y) * Lx + q.x4) =
          make_float4(e[0], e[1], e[2], e[3]);
    fm = fc;
    fc = fp;
  }
}

// ---- psi and the new phi in one z-marching kernel (Lx = 128 V, V = 1 or 2) ------
// The second and third passes of a substep fused: a CTA of F3F_NW warps owns
// F3F_NW - 2 output rows; warp w computes psi = a phih + b phi^3 - kappa
// lap phih (Eq. 36) on row y0 - 1 + w, the whole row (V float4 per lane,
// quad q of lane l at x = 128 q + 4 l, so the periodic x neighbours come from
// shuffles), and marches in z with phih of planes z, z + 1, z + 2 in
// registers.  psi goes to a four-plane shared-memory ring; after one barrier
// the inner warps form phi^{n+1} = phih + dt Gamma lap psi (Eq. 36) of plane
// z from the ring.  psi never reaches global memory: a substep moves the
// advection pass's 20 B/site plus about 12 B/site here, instead of 44 B.  The
// arithmetic runs on packed FP32 pairs.
constexpr int F3F_NW = 16;

template <int V>
__device__ __forceinline__ void xnbr_row(const float4 (&c)[V], float (&l)[V], float (&r)[V]) {
  const int lane = threadIdx.x & 31;
  float sl[V], sr[V];
#pragma unroll
  for (int q = 0; q < V; ++q) {
    sl[q] = __shfl_sync(0xffffffffu, c[q].w, (lane + 31) & 31);
    sr[q] = __shfl_sync(0xffffffffu, c[q].x, (lane + 1) & 31);
  }
#pragma unroll
  for (int q = 0; q < V; ++q) {
    l[q] = lane == 0 ? sl[(q + V - 1) % V] : sl[q];
    r[q] = lane == 31 ? sr[(q + 1) % V] : sr[q];
  }
}

// The loads of iteration z + 1 (phih of plane z + 3, phih of plane z + 2 on
// the rows y -+ 1 and phi of plane z + 2) are issued before iteration z
// computes, so that they are in flight across its barrier (1.16x over
// loading them at the top of their own iteration).
// packed FP32 pairs (sites 0,1 and 2,3 of a quad)
__device__ __forceinline__ float2 pf2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 padd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 pmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 pfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 lo2(const float4 &v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi2(const float4 &v) { return make_float2(v.z, v.w); }

// 7-point Laplacian of the quad c (x neighbours l, r of its ends; m, p in z,
// ym, yp in y) as two packed pairs: the z and y neighbours and the centre as
// pairs, the x neighbour sums (which straddle the pairs) scalar
__device__ __forceinline__ void lap7_quad(const float4 &c, const float4 &m, const float4 &p, const float4 &ym,
                                          const float4 &yp, float l, float r, float2 &lo, float2 &hi) {
  const float2 m6 = pf2(-6.f, -6.f);
  lo = pfma(m6, lo2(c), padd(padd(padd(lo2(m), lo2(p)), padd(lo2(ym), lo2(yp))), pf2(l + c.y, c.x + c.z)));
  hi = pfma(m6, hi2(c), padd(padd(padd(hi2(m), hi2(p)), padd(hi2(ym), hi2(yp))), pf2(c.y + c.w, c.z + r)));
}

template <int V, int MINB>
__global__ void __launch_bounds__(F3F_NW * 32, MINB)
    fd3f_kernel(const float *__restrict__ A, const float *__restrict__ G, float *__restrict__ out,
                KParams<float> p, int nz) {
  constexpr int NW = F3F_NW, W = 128 * V;
  extern __shared__ __align__(16) float f3f_smem[];
  float(*sq)[NW][W] = reinterpret_cast<float(*)[NW][W]>(f3f_smem);  // [4][NW][W]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int Ly = p.Ly, Lz = p.Lz;
  const long long plane = (long long)W * Ly;
  const int y0 = blockIdx.y * (NW - 2);
  const int yr = y0 - 1 + warp;  // this warp's psi row (wrapped below)
  const int y = wrapi(yr, Ly), ym = wrapi(yr - 1, Ly), yp = wrapi(yr + 1, Ly);
  const bool outw = warp >= 1 && warp <= NW - 2 && yr < Ly;  // warp-uniform
  const int z0 = blockIdx.z * nz, z1 = min(z0 + nz, Lz);
  auto rowp = [&](const float *f, int yy, int zz) { return f + wrapi(zz, Lz) * plane + (long long)yy * W; };
  auto ld = [&](const float *f, int yy, int zz, float4 (&v)[V]) {
    const float *row = rowp(f, yy, zz);
#pragma unroll
    for (int q = 0; q < V; ++q) v[q] = __ldg(reinterpret_cast<const float4 *>(row + 128 * q + 4 * lane));
  };
  auto mv = [](float4 (&d)[V], const float4 (&s2)[V]) {
#pragma unroll
    for (int q = 0; q < V; ++q) d[q] = s2[q];
  };
  float4 hm[V], hc[V], hp[V];     // phih of this row at planes z, z + 1, z + 2
  float4 hym[V], hyp[V], gc[V];   // phih of plane z + 1 on rows y -+ 1, phi of plane z + 1
  ld(A, y, z0 - 2, hm);
  ld(A, y, z0 - 1, hc);
  ld(A, y, z0, hp);
  ld(A, ym, z0 - 1, hym);
  ld(A, yp, z0 - 1, hyp);
  ld(G, y, z0 - 1, gc);
  for (int z = z0 - 2; z < z1; ++z) {
    float4 nhp[V], nym[V], nyp[V], ngc[V];
    ld(A, y, z + 3, nhp);
    ld(A, ym, z + 2, nym);
    ld(A, yp, z + 2, nyp);
    ld(G, y, z + 2, ngc);
    // psi of plane z + 1 on this warp's row
    {
      float l[V], r[V];
      xnbr_row<V>(hc, l, r);
      float *dst = &sq[(z + 1) & 3][warp][0];
#pragma unroll
      for (int q = 0; q < V; ++q) {
        float2 L[2];
        lap7_quad(hc[q], hm[q], hp[q], hym[q], hyp[q], l[q], r[q], L[0], L[1]);
        float2 o[2];
#pragma unroll
        for (int k = 0; k < 2; ++k) {
          const float2 hk = k ? hi2(hc[q]) : lo2(hc[q]);
          const float2 cb = p.cubic_at_half ? hk : (k ? hi2(gc[q]) : lo2(gc[q]));
          o[k] = pfma(pf2(p.a, p.a), hk, pfma(pf2(p.b, p.b), pmul(pmul(cb, cb), cb), pmul(pf2(-p.kappa, -p.kappa), L[k])));
        }
        *reinterpret_cast<float4 *>(dst + 128 * q + 4 * lane) = make_float4(o[0].x, o[0].y, o[1].x, o[1].y);
      }
    }
    __syncthreads();
    // phi^{n+1} of plane z (psi planes z - 1, z, z + 1 are in the ring)
    if (z >= z0 && outw) {
      auto sld = [&](int slot, int w, int q) {
        return *reinterpret_cast<const float4 *>(&sq[slot][w][128 * q + 4 * lane]);
      };
      float4 qc[V];
#pragma unroll
      for (int q = 0; q < V; ++q) qc[q] = sld(z & 3, warp, q);
      float l[V], r[V];
      xnbr_row<V>(qc, l, r);
      float *orow = out + (long long)z * plane + (long long)yr * W;
#pragma unroll
      for (int q = 0; q < V; ++q) {
        const float4 qm = sld((z + 3) & 3, warp, q), qp = sld((z + 1) & 3, warp, q);
        const float4 qym = sld(z & 3, warp - 1, q), qyp = sld(z & 3, warp + 1, q);
        float2 L[2];
        lap7_quad(qc[q], qm, qp, qym, qyp, l[q], r[q], L[0], L[1]);
        const float2 g = pf2(p.dtG, p.dtG);
        const float2 o0 = pfma(g, L[0], lo2(hm[q])), o1 = pfma(g, L[1], hi2(hm[q]));
        *reinterpret_cast<float4 *>(orow + 128 * q + 4 * lane) = make_float4(o0.x, o0.y, o1.x, o1.y);
      }
    }
    mv(hm, hc);
    mv(hc, hp);
    mv(hp, nhp);
    mv(hym, nym);
    mv(hyp, nyp);
    mv(gc, ngc);
  }
}

// ---- one whole FD substep, software-pipelined in z (Lx = 128 V, V = 1 or 2) ----
// The advection of Eqs. 32-35 fused with psi and the new phi of Eq. 36, with
// one barrier per plane.  A CTA of F3P_NW warps owns F3P_NW - 4 output rows;
// warp w owns row y0 - 2 + w, the whole row (V float4 per lane, quad q of
// lane l at x = 128 q + 4 l; periodic x neighbours by shuffles), and marches
// in z.  Iteration k runs three phases, each reading only what earlier
// iterations wrote, so that one barrier at its end orders them all:
//   C (warps 2 .. NW - 3): phi^{n+1} of plane k - 2 = phih + dt Gamma lap psi,
//     from psi of planes k - 3 .. k - 1 (three-slot ring; rows w -+ 1 of plane
//     k - 2) and phih of plane k - 2 (own row);
//   B (warps 1 .. NW - 2): psi of plane k = a phih + b phi^3 - kappa lap phih,
//     from phih of planes k - 1 .. k + 1 (four-slot ring; rows w -+ 1 of
//     plane k) into the psi ring;
//   A (all warps): phih of plane a = k + 2 into the phih ring.
// A warp writes only its own row of a ring, and the only same-iteration
// reuse of a slot is by the writing warp itself (C reads its own phih of
// plane k - 2 and psi of plane k - 3 before A and B overwrite those slots).
// The advection inputs arrive one plane ahead: u of the warps' 16 rows and v
// of 18 rows (y -+ 1) by bulk copies into a two-slot shared-memory ring (one
// mbarrier a slot; warp 0 issues plane a + 1 at the top of iteration k, after
// the barrier that ended the reads of its slot), phi and w of the own row in
// registers marching in z, and phi of rows y -+ 1 and the next planes' own-row
// phi and w loaded at the end of phase A, so that they are in flight across
// the barrier and phases C and B.  A substep reads phi and u* and writes the
// new phi (20 B/site, against 32 B/site for the advection pass followed by
// fd3f); the arithmetic per site is that of those two kernels (the same
// device functions and packed operations), so the results are equal bitwise.
// Every copy wait is bounded: a wait that gives up is reported through the
// barrier (all threads learn it together), the copies in flight are drained
// with a bound, and the CTA returns; the host reports LBM_ETIMEOUT.
constexpr int F3P_NW = 16;

__device__ int g_fd3p_err = 0;
__device__ unsigned long long g_fd3p_wait_ns = 500000000ull;

template <int V>
struct F3P {
  static constexpr int W = 128 * V;
  static constexpr int U_OFF = 0;                                // [2][NW][W]     u rows
  static constexpr int V_OFF = U_OFF + 2 * F3P_NW * W;           // [2][NW + 2][W] v rows
  static constexpr int H_OFF = V_OFF + 2 * (F3P_NW + 2) * W;     // [4][NW][W]     phih
  static constexpr int Q_OFF = H_OFF + 4 * F3P_NW * W;           // [3][NW][W]     psi
  static constexpr int FLOATS = Q_OFF + 3 * F3P_NW * W;
  static constexpr uint32_t TX_BYTES = (2 * F3P_NW + 2) * W * sizeof(float);  // one plane's copies
  static constexpr size_t smem = sizeof(float) * FLOATS + 16;    // + two mbarriers
};

template <bool FLUX, int V>
__global__ void __launch_bounds__(F3P_NW * 32, 1)
    fd3p_kernel(const float *__restrict__ G, const float *__restrict__ u, float *__restrict__ out,
                KParams<float> p, int nz) {
  constexpr int NW = F3P_NW, W = 128 * V;
  using L = F3P<V>;
  extern __shared__ __align__(16) float f3p_smem[];
  float(*su)[NW][W] = reinterpret_cast<float(*)[NW][W]>(f3p_smem + L::U_OFF);
  float(*sv)[NW + 2][W] = reinterpret_cast<float(*)[NW + 2][W]>(f3p_smem + L::V_OFF);
  float(*sh)[NW][W] = reinterpret_cast<float(*)[NW][W]>(f3p_smem + L::H_OFF);
  float(*sq)[NW][W] = reinterpret_cast<float(*)[NW][W]>(f3p_smem + L::Q_OFF);
  const uint32_t bar0 = su32(f3p_smem + L::FLOATS);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int Ly = p.Ly, Lz = p.Lz;
  const long long plane = (long long)W * Ly, Sz = plane * Lz;
  const float *vv = u + Sz, *ww = u + 2 * Sz;
  const int y0 = blockIdx.y * (NW - 4);
  const int yr = y0 - 2 + warp;  // this warp's row (wrapped below)
  const int y = wrapi(yr, Ly), ym = wrapi(yr - 1, Ly), yp = wrapi(yr + 1, Ly);
  const bool psiw = warp >= 1 && warp <= NW - 2;             // warp-uniform
  const bool outw = warp >= 2 && warp <= NW - 3 && yr < Ly;  // warp-uniform
  const int z0 = blockIdx.z * nz, z1 = min(z0 + nz, Lz);
  const int a0 = z0 - 2, a1 = z1 + 1;  // planes phase A advects
  const bool cubic_half = p.cubic_at_half != 0;
  auto g4 = [&](const float *f, int yy, int zz, int q) {
    return __ldg(reinterpret_cast<const float4 *>(f + wrapi(zz, Lz) * plane + (long long)yy * W + 128 * q +
                                                  4 * lane));
  };
  auto ldrow = [&](const float *f, int yy, int zz, float4(&v)[V]) {
#pragma unroll
    for (int q = 0; q < V; ++q) v[q] = g4(f, yy, zz, q);
  };
  auto put = [&](float(*ring)[NW][W], int slot, const float4(&v)[V]) {
#pragma unroll
    for (int q = 0; q < V; ++q) *reinterpret_cast<float4 *>(&ring[slot][warp][128 * q + 4 * lane]) = v[q];
  };
  auto get = [&](const float *row, int q) { return *reinterpret_cast<const float4 *>(row + 128 * q + 4 * lane); };
  // u and v rows of plane pl (warp 0): 16 + 18 bulk copies of one row each
  auto issue = [&](int pl) {
    const int s = pl & 1;
    const uint32_t bar = bar0 + 8 * s;
    if (lane == 0) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // earlier reads of the slot first
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(L::TX_BYTES)
                   : "memory");
    }
    __syncwarp();
    const long long zo = (long long)wrapi(pl, Lz) * plane;
    for (int i = lane; i < 2 * NW + 2; i += 32) {
      const float *src;
      uint32_t dst;
      if (i < NW) {
        src = u + zo + (long long)wrapi(y0 - 2 + i, Ly) * W;
        dst = su32(&su[s][i][0]);
      } else {
        src = vv + zo + (long long)wrapi(y0 - 3 + (i - NW), Ly) * W;
        dst = su32(&sv[s][i - NW][0]);
      }
      asm volatile(
          "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
          "l"(src), "r"((uint32_t)(W * sizeof(float))), "r"(bar)
          : "memory");
    }
  };
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0 + 8) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (warp == 0) {
    issue(a0);
    if (a0 + 1 <= a1) issue(a0 + 1);
  }
  // own-row phi of planes a - 1, a, a + 1 and w of the same (a = the plane
  // phase A advects next), phi of plane a on rows y -+ 1, and phi of plane k
  // (the cube of phase B)
  float4 P0[V], P1[V], P2[V], Pym[V], Pyp[V], W0[V], W1[V], W2[V], Pk[V];
  ldrow(G, y, a0 - 1, P0);
  ldrow(G, y, a0, P1);
  ldrow(G, y, a0 + 1, P2);
  ldrow(G, ym, a0, Pym);
  ldrow(G, yp, a0, Pyp);
  ldrow(ww, y, a0 - 1, W0);
  ldrow(ww, y, a0, W1);
  ldrow(ww, y, a0 + 1, W2);
#pragma unroll
  for (int q = 0; q < V; ++q) Pk[q] = make_float4(0.f, 0.f, 0.f, 0.f);
  const float2 g2 = pf2(p.dtG, p.dtG);
  for (int k = z0 - 4; k <= z1 + 1; ++k) {
    if (warp == 0 && k >= z0 - 3 && k + 3 <= a1) issue(k + 3);
    // C: phi^{n+1} of plane k - 2
    if (k >= z0 + 2 && outw) {
      const int zc = k - 2;
      const float *qrow = &sq[(zc + 6) % 3][warp][0];
      float4 qc[V];
#pragma unroll
      for (int q = 0; q < V; ++q) qc[q] = get(qrow, q);
      float l[V], r[V];
      xnbr_row<V>(qc, l, r);
      float *orow = out + (long long)zc * plane + (long long)yr * W;
#pragma unroll
      for (int q = 0; q < V; ++q) {
        const float4 qm = get(&sq[(zc + 5) % 3][warp][0], q), qp = get(&sq[(zc + 7) % 3][warp][0], q);
        const float4 qym = get(&sq[(zc + 6) % 3][warp - 1][0], q), qyp = get(&sq[(zc + 6) % 3][warp + 1][0], q);
        const float4 hm = get(&sh[zc & 3][warp][0], q);
        float2 Lp[2];
        lap7_quad(qc[q], qm, qp, qym, qyp, l[q], r[q], Lp[0], Lp[1]);
        const float2 o0 = pfma(g2, Lp[0], lo2(hm)), o1 = pfma(g2, Lp[1], hi2(hm));
        *reinterpret_cast<float4 *>(orow + 128 * q + 4 * lane) = make_float4(o0.x, o0.y, o1.x, o1.y);
      }
    }
    // B: psi of plane k
    if (k >= z0 - 1 && k <= z1 && psiw) {
      float4 hc[V];
#pragma unroll
      for (int q = 0; q < V; ++q) hc[q] = get(&sh[k & 3][warp][0], q);
      float l[V], r[V];
      xnbr_row<V>(hc, l, r);
      float4 o4[V];
#pragma unroll
      for (int q = 0; q < V; ++q) {
        const float4 hm = get(&sh[(k + 3) & 3][warp][0], q), hp = get(&sh[(k + 1) & 3][warp][0], q);
        const float4 hym = get(&sh[k & 3][warp - 1][0], q), hyp = get(&sh[k & 3][warp + 1][0], q);
        float2 Lp[2];
        lap7_quad(hc[q], hm, hp, hym, hyp, l[q], r[q], Lp[0], Lp[1]);
        float2 o[2];
#pragma unroll
        for (int kk = 0; kk < 2; ++kk) {
          const float2 hk = kk ? hi2(hc[q]) : lo2(hc[q]);
          const float2 cb = cubic_half ? hk : (kk ? hi2(Pk[q]) : lo2(Pk[q]));
          o[kk] = pfma(pf2(p.a, p.a), hk,
                       pfma(pf2(p.b, p.b), pmul(pmul(cb, cb), cb), pmul(pf2(-p.kappa, -p.kappa), Lp[kk])));
        }
        o4[q] = make_float4(o[0].x, o[0].y, o[1].x, o[1].y);
      }
      put(sq, (k + 6) % 3, o4);
    }
    // A: phih of plane a = k + 2, then the loads of plane a + 1
    bool ok = true;
    const int a = k + 2;
    if (a <= a1) {
      const int s = a & 1;
      ok = bar_wait(bar0 + 8 * s, (uint32_t)((a - a0) >> 1) & 1u, g_fd3p_wait_ns);
      float4 uc[V];
#pragma unroll
      for (int q = 0; q < V; ++q) uc[q] = get(&su[s][warp][0], q);
      float pl[V], pr[V], ul[V], ur[V];
      xnbr_row<V>(P1, pl, pr);
      xnbr_row<V>(uc, ul, ur);
      float4 h[V];
#pragma unroll
      for (int q = 0; q < V; ++q) {
        const float4 vc = get(&sv[s][warp + 1][0], q), vym = get(&sv[s][warp][0], q),
                     vyp = get(&sv[s][warp + 2][0], q);
        float e[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const float ph = cmp4(P1[q], j);
          const float pxm = j == 0 ? pl[q] : cmp4(P1[q], j - 1), pxp = j == 3 ? pr[q] : cmp4(P1[q], j + 1);
          const float uxm = j == 0 ? ul[q] : cmp4(uc[q], j - 1), uxp = j == 3 ? ur[q] : cmp4(uc[q], j + 1);
          e[j] = adv_site<FLUX>(ph, pxm, pxp, cmp4(Pym[q], j), cmp4(Pyp[q], j), cmp4(P0[q], j), cmp4(P2[q], j),
                                uxm, cmp4(uc[q], j), uxp, cmp4(vym, j), cmp4(vc, j), cmp4(vyp, j),
                                cmp4(W0[q], j), cmp4(W1[q], j), cmp4(W2[q], j), p.dt);
        }
        h[q] = make_float4(e[0], e[1], e[2], e[3]);
      }
      put(sh, a & 3, h);
      // march: phi of plane a - 1 becomes the cube of the next phase B
#pragma unroll
      for (int q = 0; q < V; ++q) {
        Pk[q] = P0[q];
        P0[q] = P1[q];
        P1[q] = P2[q];
        W0[q] = W1[q];
        W1[q] = W2[q];
      }
      if (a + 1 <= a1) {
        ldrow(G, y, a + 2, P2);
        ldrow(G, ym, a + 1, Pym);
        ldrow(G, yp, a + 1, Pyp);
        ldrow(ww, y, a + 2, W2);
      }
    } else {
      // no plane left to advect: phi of plane k + 1 for the last phase B
#pragma unroll
      for (int q = 0; q < V; ++q) {
        Pk[q] = P0[q];
        P0[q] = P1[q];
      }
    }
    if (!__syncthreads_and(ok)) {
      // a copy did not land within the bound: report, drain what is in
      // flight (planes a and a + 1, with the 0.5 s bound), leave
      if (threadIdx.x == 0) {
        atomicExch(&g_fd3p_err, 1);
        for (int pl = a; pl <= min(a + 1, a1); ++pl)
          bar_wait(bar0 + 8 * (pl & 1), (uint32_t)((pl - a0) >> 1) & 1u, 500000000ull);
      }
      return;
    }
  }
}

// resident CTAs of the pipelined substep kernel on this device (queried once per V)
template <int V>
int fd3p_resident_v() {
  static const int g = [] {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fd3p_kernel<false, V>, F3P_NW * 32, F3P<V>::smem);
    return std::max(1, sms * std::max(per, 1));
  }();
  return g;
}

template <typename S, typename C>
__global__ void __launch_bounds__(256)
    density3d_kernel(const S *__restrict__ hin, C *__restrict__ dn, KParams<C> p) {
  const int Lx = p.Lx, Ly = p.Ly, Lz = p.Lz;
  const long long Sz = (long long)Lx * Ly * Lz;
  const int x = blockIdx.x * 32 + threadIdx.x, y = blockIdx.y * 8 + threadIdx.y, z = blockIdx.z;
  if (x >= Lx || y >= Ly) return;
  C d = C(0);
#pragma unroll
  for (int i = 0; i < 19; ++i) {
    const int sx = wrapi(x - q19_ex(i), Lx), sy = wrapi(y - q19_ey(i), Ly),
              sz = wrapi(z - q19_ez(i), Lz);
    d += Store<S, C>::ld(hin + i * Sz + ((long long)sz * Ly + sy) * Lx + sx, p.inv_scale);
  }
  dn[((long long)z * Ly + y) * Lx + x] = d;
}

template <typename S, typename C>
cudaError_t collide3d(lbm_handle *h, int in, int force_on, int mode) {
  KParams<C> p = make_params<C>(h, force_on);
  dim3 grid((p.Lx + C3_TX - 1) / C3_TX, (p.Ly + C3_TY - 1) / C3_TY, (p.Lz + c3_tz<C>() - 1) / c3_tz<C>());
  dim3 block(32, C3_TY);
  const S *hin = static_cast<const S *>(h->h[in]);
  S *hout = static_cast<S *>(h->h[1 - in]);
  const C *phi = static_cast<const C *>(h->phi[in]);
  const C *dn = static_cast<const C *>(h->dn);
  C *u = static_cast<C *>(h->u);
  const bool tgen = p.cs2mT != C(0);
  // registers budgeted for 3 CTAs per SM (85 a thread, no spill in FP32): 576 us
  // at 256^3 against 698 us for 2 and 618 us for 4 (spilling)
  if (mode == COLLIDE_STEP) {
    if (tgen)
      collide3d_kernel<S, C, true, COLLIDE_STEP, 3><<<grid, block, 0, h->stream>>>(hin, hout, phi, dn, u, h->staging, p);
    else
      collide3d_kernel<S, C, false, COLLIDE_STEP, 3><<<grid, block, 0, h->stream>>>(hin, hout, phi, dn, u, h->staging, p);
  } else {
    if (tgen)
      collide3d_kernel<S, C, true, COLLIDE_MOMENTS, 3><<<grid, block, 0, h->stream>>>(hin, hout, phi, dn, u, h->staging, p);
    else
      collide3d_kernel<S, C, false, COLLIDE_MOMENTS, 3><<<grid, block, 0, h->stream>>>(hin, hout, phi, dn, u, h->staging, p);
  }
  return cudaGetLastError();
}

// resident blocks of the advection pass on this device (queried once per form)
template <bool FLUX>
long long f3v_resident() {
  static const long long g = [] {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fd3v_adv_kernel<FLUX>, 256, 0);
    return (long long)std::max(1, sms * std::max(per, 1));
  }();
  return g;
}

// the m substeps of an LB step as three passes each (FP32)
cudaError_t fd3d_passes(lbm_handle *h, int in) {
  KParams<float> p = make_params<float>(h, 0);
  dim3 grid((p.Lx + 31) / 32, (p.Ly + 7) / 8, p.Lz), block(32, 8);
  const float *u = static_cast<const float *>(h->u);
  float *A = static_cast<float *>(h->fd_a), *P = static_cast<float *>(h->fd_p);
  const float *src = static_cast<const float *>(h->phi[in]);
  const bool flux = p.adv_variant == LBM_ADV_FLUX;
  const bool vec = p.Lx % 4 == 0 && p.Lx >= 4 && std::getenv("HLBM_FD3_SCALAR") == nullptr;
  // planes per thread (at most F3V_NZ): the kernels run a few waves of
  // resident blocks, and a partial last wave leaves most SMs idle while its
  // blocks march their planes, so nz minimises waves x (nz + 2), the planes a
  // block loads (its first two are the z neighbours of the first output)
  const long long bxy = (long long)((p.Lx / 4 + 31) / 32) * ((p.Ly + 7) / 8);
  const long long res = flux ? f3v_resident<true>() : f3v_resident<false>();
  int nz = 1;
  long long best = -1;
  for (int c = 1; c <= std::min(F3V_NZ, p.Lz); ++c) {
    const long long waves = (bxy * ((p.Lz + c - 1) / c) + res - 1) / res;
    if (best < 0 || waves * (c + 2) < best) {
      best = waves * (c + 2);
      nz = c;
    }
  }
  dim3 gridv((p.Lx / 4 + 31) / 32, (p.Ly + 7) / 8, (p.Lz + nz - 1) / nz);
  // psi and the new phi fused (whole rows per warp: Lx = 128 or 256); planes
  // per CTA: about two (Lx = 128) or one (Lx = 256, 128 registers a thread)
  // CTAs per SM of 152, at least 4
  const bool fused = vec && (p.Lx == 128 || p.Lx == 256) && std::getenv("HLBM_FD3_UNFUSED") == nullptr;
  const int rows_f = (p.Ly + F3F_NW - 3) / (F3F_NW - 2);
  const int nzf = std::max(4, std::min(p.Lz, (int)((long long)p.Lz * rows_f / 304)));
  dim3 gridf(1, rows_f, (p.Lz + nzf - 1) / nzf);
  const int nzf1 = std::max(4, std::min(p.Lz, (int)((long long)p.Lz * rows_f / 152)));  // one CTA per SM
  dim3 gridf1(1, rows_f, (p.Lz + nzf1 - 1) / nzf1);
  // the advection fused as well, one software-pipelined kernel per substep
  // (opt-in; one CTA per SM, within one wave of z chunks)
  const bool fusedp = fused && std::getenv("HLBM_FD3_FUSED_ADV") != nullptr;
  const int rows_p = (p.Ly + F3P_NW - 5) / (F3P_NW - 4);
  const int zch = std::max(1, std::min(p.Lz, (p.Lx == 128 ? fd3p_resident_v<1>() : fd3p_resident_v<2>()) / rows_p));
  const int nzp = (p.Lz + zch - 1) / zch;
  dim3 gridp(1, rows_p, (p.Lz + nzp - 1) / nzp);
  for (int j = 0; j < h->m; ++j) {
    float *dst = static_cast<float *>(((h->m - 1 - j) % 2 == 0) ? h->phi[1 - in] : h->phi[2]);
    if (fusedp) {
      if (p.Lx == 128) {
        if (flux) fd3p_kernel<true, 1><<<gridp, F3P_NW * 32, F3P<1>::smem, h->stream>>>(src, u, dst, p, nzp);
        else fd3p_kernel<false, 1><<<gridp, F3P_NW * 32, F3P<1>::smem, h->stream>>>(src, u, dst, p, nzp);
      } else {
        if (flux) fd3p_kernel<true, 2><<<gridp, F3P_NW * 32, F3P<2>::smem, h->stream>>>(src, u, dst, p, nzp);
        else fd3p_kernel<false, 2><<<gridp, F3P_NW * 32, F3P<2>::smem, h->stream>>>(src, u, dst, p, nzp);
      }
    } else if (vec) {
      if (flux) fd3v_adv_kernel<true><<<gridv, block, 0, h->stream>>>(src, u, A, p, nz);
      else fd3v_adv_kernel<false><<<gridv, block, 0, h->stream>>>(src, u, A, p, nz);
      if (fused) {
        const size_t smf = sizeof(float) * 4 * F3F_NW * p.Lx;
        if (p.Lx == 128) fd3f_kernel<1, 2><<<gridf, F3F_NW * 32, smf, h->stream>>>(A, src, dst, p, nzf);
        else fd3f_kernel<2, 1><<<gridf1, F3F_NW * 32, smf, h->stream>>>(A, src, dst, p, nzf1);
      } else {
        fd3v_lap_kernel<true><<<gridv, block, 0, h->stream>>>(A, src, P, p, nz);
        fd3v_lap_kernel<false><<<gridv, block, 0, h->stream>>>(P, A, dst, p, nz);
      }
    } else {
      if (flux) fd3_adv_kernel<true><<<grid, block, 0, h->stream>>>(src, u, A, p);
      else fd3_adv_kernel<false><<<grid, block, 0, h->stream>>>(src, u, A, p);
      fd3_psi_kernel<<<grid, block, 0, h->stream>>>(A, src, P, p);
      fd3_phi_kernel<<<grid, block, 0, h->stream>>>(P, A, dst, p);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    src = dst;
  }
  return cudaSuccess;
}

template <typename C, int TX, int TY, int TZ>
cudaError_t fd3d(lbm_handle *h, int in) {
  KParams<C> p = make_params<C>(h, 0);
  dim3 grid((p.Lx + TX - 1) / TX, (p.Ly + TY - 1) / TY, (p.Lz + TZ - 1) / TZ), block(32, 8);
  const int launches = (h->m + h->sub - 1) / h->sub;
  const C *u = static_cast<const C *>(h->u);
  const C *src = static_cast<const C *>(h->phi[in]);
  for (int j = 0; j < launches; ++j) {
    const int sub = (j == launches - 1) ? h->m - h->sub * (launches - 1) : h->sub;
    C *dst = static_cast<C *>(((launches - 1 - j) % 2 == 0) ? h->phi[1 - in] : h->phi[2]);
    const int H = 3 * sub;
    const size_t smem = sizeof(C) * 6 * (size_t)(TX + 2 * H) * (TY + 2 * H) * (TZ + 2 * H);
    fd3d_kernel<C, TX, TY, TZ><<<grid, block, smem, h->stream>>>(src, u, dst, p, sub);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    src = dst;
  }
  return cudaSuccess;
}

}  // namespace

// FD tiles: FP32 32 x 4 x 4, FP64 16 x 4 x 4 (one substep per launch: halo 3).
constexpr int FD3_TX_F = 32, FD3_TX_D = 16, FD3_TY = 4, FD3_TZ = 4;

size_t fd3d_smem_bytes(int precision, int sub) {
  const int H = 3 * sub;
  const int tx = precision == LBM_F64 ? FD3_TX_D : FD3_TX_F;
  const size_t cb = precision == LBM_F64 ? 8 : 4;
  return cb * 6 * (size_t)(tx + 2 * H) * (FD3_TY + 2 * H) * (FD3_TZ + 2 * H);
}

cudaError_t fd3d_configure(int precision, size_t smem) {
  if (precision == LBM_F64)
    return cudaFuncSetAttribute(fd3d_kernel<double, FD3_TX_D, FD3_TY, FD3_TZ>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  cudaError_t e = cudaFuncSetAttribute(fd3d_kernel<float, FD3_TX_F, FD3_TY, FD3_TZ>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(fd3f_kernel<1, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(sizeof(float) * 4 * F3F_NW * 128));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(fd3f_kernel<2, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(sizeof(float) * 4 * F3F_NW * 256));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(fd3p_kernel<false, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)F3P<1>::smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(fd3p_kernel<true, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)F3P<1>::smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(fd3p_kernel<false, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)F3P<2>::smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(fd3p_kernel<true, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)F3P<2>::smem);
  return e;
}

int fd3p_set_wait_ns(unsigned long long ns) {
  return cudaMemcpyToSymbol(g_fd3p_wait_ns, &ns, sizeof ns) == cudaSuccess ? 0 : -1;
}

int fd3p_error(bool reset) {
  int v = 0;
  if (cudaMemcpyFromSymbol(&v, g_fd3p_err, sizeof v) != cudaSuccess) return -1;
  if (reset && v != 0) {
    const int zero = 0;
    cudaMemcpyToSymbol(g_fd3p_err, &zero, sizeof zero);
  }
  return v;
}

cudaError_t collide3d_launch(lbm_handle *h, int in, int force_on, int mode) {
  switch (h->P.precision) {
    case LBM_F64: return collide3d<double, double>(h, in, force_on, mode);
    case LBM_F32DEV: return collide3d<float, float>(h, in, force_on, mode);
    default: return collide3d<__half, float>(h, in, force_on, mode);
  }
}

cudaError_t fd3d_launch(lbm_handle *h, int in) {
  if (h->P.precision == LBM_F64) return fd3d<double, FD3_TX_D, FD3_TY, FD3_TZ>(h, in);
  if (h->fd_a != nullptr && std::getenv("HLBM_FD3_TILE") == nullptr) return fd3d_passes(h, in);
  return fd3d<float, FD3_TX_F, FD3_TY, FD3_TZ>(h, in);
}

cudaError_t density3d_launch(lbm_handle *h, int in) {
  dim3 grid((h->P.Lx + 31) / 32, (h->P.Ly + 7) / 8, h->P.Lz), block(32, 8);
  switch (h->P.precision) {
    case LBM_F64: {
      KParams<double> p = make_params<double>(h, 0);
      density3d_kernel<double, double><<<grid, block, 0, h->stream>>>(
          static_cast<const double *>(h->h[in]), static_cast<double *>(h->dn), p);
      break;
    }
    case LBM_F32DEV: {
      KParams<float> p = make_params<float>(h, 0);
      density3d_kernel<float, float><<<grid, block, 0, h->stream>>>(
          static_cast<const float *>(h->h[in]), static_cast<float *>(h->dn), p);
      break;
    }
    default: {
      KParams<float> p = make_params<float>(h, 0);
      density3d_kernel<__half, float><<<grid, block, 0, h->stream>>>(
          static_cast<const __half *>(h->h[in]), static_cast<float *>(h->dn), p);
    }
  }
  return cudaGetLastError();
}

}  // namespace hlbm
