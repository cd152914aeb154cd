// One leapfrog step of the cut-cell model on the GPU (paper Sec 2.2 and 2.4).
//
//   k_full   every interior cell and corner of every (domain, tile) work item:
//            scalar fluxes and divergence with full apertures (Eq. fvm_d), the
//            p' and rho' tendencies, momentum on regular velocity cells
//            (Eqs. momentum_u_d .. w_d), fourth-order diffusion, sponge,
//            leapfrog and Robert-Asselin filter.  A 2.5D march in z keeps
//            rings of haloed planes in shared memory, filled by asynchronous
//            copies (cp.async) issued three planes ahead of the work; two
//            barriers per plane.  The
//            periodic lateral boundary (Sec 3) is folded into the per-thread
//            load offsets, so no ghost exchange is needed.  Branch-free: cut
//            cells and diagnosed corners are recomputed by the list kernels.
//   k_groups one thread per merge group / cut cell: face fluxes weighted by
//            the apertures, divergence over the merged volume, host update
//            and scatter to the absorbed cells (Sec 2.3, 2.4).
//   k_diag   one thread per column: boundary velocity by the nearest-plane
//            interpolation and free-slip projection (Eq. 33), merged-face
//            interpolation, lid values, the values below the terrain.
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>

#include "cc_internal.h"

namespace cc {

// ------------------------------------------------------------------ arithmetic
template <typename T>
struct Ar;
template <>
struct Ar<double> {
  static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
  static __device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
  static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
};
template <>
struct Ar<float> {
  static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
  static __device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
  static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
};

// Face flux phi_f * u_n * S with phi_f the mean of the two cells (lower index
// first) and u_n the mean of the four corner values, summed pairwise.  Every
// operation is rounded as written, so a face evaluated from either side, or
// by either kernel, gives the same bits and cancels exactly in the sum.
template <typename T>
__device__ __forceinline__ T face_flux(T pa, T pb, T u1, T u2, T u3, T u4, T S) {
  using A = Ar<T>;
  T un = A::mul(A::add(A::add(u1, u2), A::add(u3, u4)), T(0.25));
  return A::mul(A::mul(A::mul(A::add(pa, pb), T(0.5)), un), S);
}

// Corner density: mean of the eight surrounding cell totals (dk outer, then
// dj, then di; -1 before 0), summed pairwise.
template <typename T>
__device__ __forceinline__ T rho8(T a, T b, T c, T d, T e, T f, T g, T h) {
  using A = Ar<T>;
  return A::mul(A::add(A::add(A::add(a, b), A::add(c, d)), A::add(A::add(e, f), A::add(g, h))), T(0.125));
}

// reciprocal of the corner density; the velocity is momentum times it.
// FP32: the hardware reciprocal approximation (relative error below 2^-22,
// under the FP32 form's other rounding); every kernel uses this same function,
// so a corner velocity has the same bits in each
__device__ __forceinline__ double rinv(double rc) { return 1.0 / rc; }
__device__ __forceinline__ float rinv(float rc) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(rc));
  return r;
}

// rho*theta as a function of pressure (equation of state, Sec 2.1:
// rho theta = (p0/R)(p/p0)^(cv/cp)) and the Exner-type factor (p/p0)^(R/cp),
// both about the per-level base values: with x = p'/p_bar,
// (rho theta)' = (rho theta)_bar ((1 + x)^(cv/cp) - 1) and the Exner factor
// pi_bar (1 + ((1 + x)^(R/cp) - 1)).  FP64: (1 + x)^a - 1 as the binomial
// series sum_{n=1..12} C(a, n) x^n for |x| < 1/32 (truncation below 1e-17
// relative), else through log1p / expm1; a resting state gives exactly zero.
__device__ __forceinline__ double pow1pm1(double x, const double *c) {
  if (fabs(x) < 0.03125) {
    double s = c[11];
#pragma unroll
    for (int n = 10; n >= 0; n--) s = fma(s, x, c[n]);
    return __dmul_rn(s, x);
  }
  return expm1(__dmul_rn(c[12], log1p(x)));
}
__device__ __forceinline__ double theta_pert(const DomDev &D, const double *thb, const double *pb,
                                             const double *ipb, int kp, double pp) {
  return __dmul_rn(thb[kp], pow1pm1(__dmul_rn(pp, ipb[kp]), D.dsth));
}
__device__ __forceinline__ double theta_tot(const DomDev &D, const double *thb, const double *pb,
                                            const double *ipb, int kp, double pp) {
  return __dadd_rn(thb[kp], theta_pert(D, thb, pb, ipb, kp, pp));
}
__device__ __forceinline__ double exner_fac(const DomDev &D, const double *pik, const double *pb,
                                            const double *ipb, int kp, double pp) {
  return fma(pik[kp], pow1pm1(__dmul_rn(pp, ipb[kp]), D.dsex), pik[kp]);
}
// FP32 perturbation form: with x = p'/p_bar, (1 + x)^a - 1 is summed as the
// binomial series sum_{n=1..7} C(a, n) x^n for |x| < 1/16 (truncation below
// 1e-10 relative), else through log1p / expm1.  Every step uses an explicit
// fused multiply-add or a rounded operation, so all kernels agree bitwise.
__device__ __forceinline__ float pow1pm1(float x, const float *c) {
  if (fabsf(x) < 0.0625f) {
    float s = c[6];
    s = fmaf(s, x, c[5]);
    s = fmaf(s, x, c[4]);
    s = fmaf(s, x, c[3]);
    s = fmaf(s, x, c[2]);
    s = fmaf(s, x, c[1]);
    s = fmaf(s, x, c[0]);
    return __fmul_rn(s, x);
  }
  return expm1f(__fmul_rn(c[7], log1pf(x)));
}
__device__ __forceinline__ float theta_pert(const DomDev &D, const float *thb, const float *pb,
                                            const float *ipb, int kp, float pp) {
  return __fmul_rn(thb[kp], pow1pm1(__fmul_rn(pp, ipb[kp]), D.sth));
}
__device__ __forceinline__ float theta_tot(const DomDev &D, const float *thb, const float *pb,
                                           const float *ipb, int kp, float pp) {
  return __fadd_rn(thb[kp], theta_pert(D, thb, pb, ipb, kp, pp));
}
__device__ __forceinline__ float exner_fac(const DomDev &D, const float *pik, const float *pb,
                                           const float *ipb, int kp, float pp) {
  return fmaf(pik[kp], pow1pm1(__fmul_rn(pp, ipb[kp]), D.sex), pik[kp]);
}

// (1 + x)^a - 1 away from zero: rare, kept out of line so that the stencils'
// loops stay small
__device__ __noinline__ float pow1pm1_far(float x, float a) { return expm1f(__fmul_rn(a, log1pf(x))); }
// The same equation-of-state operations on per-level base values already in
// registers and on coefficients passed as kernel parameters (constant bank):
// bit-identical to the functions above.
__device__ __forceinline__ float pow1pm1_e(float x, const float (&c)[8]) {
  if (fabsf(x) < 0.0625f) {
    float s = c[6];
    s = fmaf(s, x, c[5]);
    s = fmaf(s, x, c[4]);
    s = fmaf(s, x, c[3]);
    s = fmaf(s, x, c[2]);
    s = fmaf(s, x, c[1]);
    s = fmaf(s, x, c[0]);
    return __fmul_rn(s, x);
  }
  return pow1pm1_far(x, c[7]);
}
__device__ __forceinline__ float theta_pert_e(const Eos &E, float thb, float ipb, float pp) {
  return __fmul_rn(thb, pow1pm1_e(__fmul_rn(pp, ipb), E.sth));
}
__device__ __forceinline__ float theta_tot_e(const Eos &E, float thb, float ipb, float pp) {
  return __fadd_rn(thb, theta_pert_e(E, thb, ipb, pp));
}
__device__ __forceinline__ float exner_e(const Eos &E, float pik, float ipb, float pp) {
  return fmaf(pik, pow1pm1_e(__fmul_rn(pp, ipb), E.sex), pik);
}
__device__ __forceinline__ double pow1pm1_e(double x, const double (&c)[13]) {
  if (fabs(x) < 0.03125) {
    double s = c[11];
#pragma unroll
    for (int n = 10; n >= 0; n--) s = fma(s, x, c[n]);
    return __dmul_rn(s, x);
  }
  return expm1(__dmul_rn(c[12], log1p(x)));
}
__device__ __forceinline__ double theta_pert_e(const Eos &E, double thb, double ipb, double pp) {
  return __dmul_rn(thb, pow1pm1_e(__dmul_rn(pp, ipb), E.dsth));
}
__device__ __forceinline__ double theta_tot_e(const Eos &E, double thb, double ipb, double pp) {
  return __dadd_rn(thb, theta_pert_e(E, thb, ipb, pp));
}
__device__ __forceinline__ double exner_e(const Eos &E, double pik, double ipb, double pp) {
  return fma(pik, pow1pm1_e(__dmul_rn(pp, ipb), E.dsex), pik);
}
// per-precision adapters of one cell level kp
template <typename T>
struct EosK;
template <>
struct EosK<float> {
  float thb, ipb, pik;
  __device__ __forceinline__ void load(const float *thb_, const float *pb_, const float *ipb_, const float *pik_,
                                       int kp) {
    thb = thb_[kp];
    ipb = ipb_[kp];
    pik = pik_[kp];
  }
  __device__ __forceinline__ float tot(const Eos &E, float pp) const { return theta_tot_e(E, thb, ipb, pp); }
  __device__ __forceinline__ float pert(const Eos &E, float pp) const { return theta_pert_e(E, thb, ipb, pp); }
  __device__ __forceinline__ float exner(const Eos &E, float pp) const { return exner_e(E, pik, ipb, pp); }
};
template <>
struct EosK<double> {
  double thb, ipb, pik;
  __device__ __forceinline__ void load(const double *thb_, const double *pb_, const double *ipb_,
                                       const double *pik_, int kp) {
    thb = thb_[kp];
    ipb = ipb_[kp];
    pik = pik_[kp];
  }
  __device__ __forceinline__ double tot(const Eos &E, double pp) const { return theta_tot_e(E, thb, ipb, pp); }
  __device__ __forceinline__ double pert(const Eos &E, double pp) const { return theta_pert_e(E, thb, ipb, pp); }
  __device__ __forceinline__ double exner(const Eos &E, double pp) const { return exner_e(E, pik, ipb, pp); }
};

__device__ __forceinline__ double d4(double a, double b, double c, double d, double e) {
  return a - 4.0 * b + 6.0 * c - 4.0 * d + e;
}
__device__ __forceinline__ float d4(float a, float b, float c, float d, float e) {
  return a - 4.0f * b + 6.0f * c - 4.0f * d + e;
}

// Artificial diffusion along one axis (Sec 2.1: fourth order; Sec 2.4: a
// second-order term where the neighbouring fluid points the fourth-order term
// needs are missing, with the boundary conditions of the terrain surface;
// reading C-4), as the axis's term of the sum S in D = -K4 S: the fourth
// difference where the neighbours at distance 1 and 2 (flags fa, fb, fd, fe)
// are all fluid points, otherwise -4 times the second difference over the
// distance-1 neighbours (K2 = 4 K4 / d^2).  A scalar neighbour that is not a
// fluid point takes the centre value (no flux through the wall); a velocity
// neighbour keeps its stored boundary value.
template <typename T>
__device__ __forceinline__ T diff_axis(T a, T b, T c, T d, T e, bool fa, bool fb, bool fd, bool fe,
                                       bool scalar) {
  if (fa && fb && fd && fe) return d4(a, b, c, d, e);
  const T lo = (fb || !scalar) ? b : c;
  const T hi = (fd || !scalar) ? d : c;
  return T(-4) * ((lo - T(2) * c) + hi);
}
__device__ __forceinline__ bool fluid_at(int k, int lo, int top) { return k >= lo && k < top; }

// padded index of a cell / corner; periodic domains wrap the lateral
// coordinates, refined boxes read their ghost frame
__device__ __forceinline__ long long widx(const DomDev &D, int i, int j, int k) {
  return D.periodic ? pidx(D, wrapi(i, D.nx), wrapi(j, D.ny), k) : pidx(D, i, j, k);
}

// ------------------------------------------------------------------ base state
// Hydrostatic base state of constant N on every padded level, evaluated in
// FP64 and stored in the model precision.
template <typename T>
__global__ void k_base(DomDev D, double theta0, double N, double p_surf, double sponge_frac,
                       double tau_max, T *rhob, T *pb, T *thb, T *pik, T *rhobc, T *tau, T *ipb) {
  int kp = blockIdx.x * blockDim.x + threadIdx.x;
  if (kp >= D.pz) return;
  auto base = [&](double z, double &rho, double &p) {
    double pis = pow(p_surf / D.p0, D.kap);
    double th, pi;
    if (N > 0.0) {
      double n2g = N * N / D.g;
      th = theta0 * exp(n2g * z);
      pi = pis + D.g * D.g / (D.cp * theta0 * N * N) * (exp(-n2g * z) - 1.0);
    } else {
      th = theta0;
      pi = pis - D.g * z / (D.cp * theta0);
    }
    p = D.p0 * pow(pi, D.cp / D.R);
    rho = p / (D.R * th * pi);
  };
  int k = kp - GH;
  double r, p, rm, pm;
  base((k + 0.5) * D.dz, r, p);
  base((k - 0.5) * D.dz, rm, pm);
  rhob[kp] = (T)r;
  pb[kp] = (T)p;
  ipb[kp] = (T)(1.0 / p);
  thb[kp] = (T)__dmul_rn(D.p0 / D.R, pow(p / D.p0, D.cvcp));
  pik[kp] = (T)pow(p / D.p0, D.kap);
  // corner level K = k: mean of the two adjacent cell levels
  rhobc[kp] = (T)(0.5 * (rm + r));
  double ztop = D.ztop, zs = ztop * (1.0 - sponge_frac), z = k * D.dz, t = 0.0;
  if (sponge_frac > 0.0 && z > zs && z <= ztop) {
    double s = sin(0.5 * M_PI * (z - zs) / (ztop - zs));
    t = tau_max * s * s;
  }
  tau[kp] = (T)t;
}

// ------------------------------------------------------------------ full-cell stencil
template <typename T, int TYv>
struct FullCfg {
  static constexpr int TX = TILE_X, TY = TYv, NT = TX * TY, HX = TX + 4, HY = TY + 4, PL = HX * HY,
                       NLP = (PL + NT - 1) / NT;
};

// Shared-memory rings of haloed planes.  Raw planes arrive by asynchronous
// copies issued three planes ahead (after the barrier that ends the previous
// plane, so a slot is rewritten only once no thread reads it); derived planes
// (total density, total rho theta, corner velocity) are formed one plane ahead
// of their use.  Each ring holds exactly the planes still read at plane k.
template <typename T, int PLn>
struct FullSmem {
  T cr[5][PLn], cp[5][PLn];  // raw rho', p' (current level), planes k-1 .. k+3
  T cm[4][3][PLn];           // raw momentum (current level), planes k-1 .. k+2 (+ in flight)
  T op[4][PLn];              // raw p' at n-1, planes k .. k+3
  T om[4][3][PLn];           // raw momentum at n-1, planes k .. k+3
  T rh[4][PLn], th[4][PLn];  // total density and total rho theta, planes k-1 .. k+2
  T uu[3][3][PLn];           // corner velocity, planes k-1 .. k+1
  T to[PLn];                 // (rho theta)' at n-1, plane k
};

__device__ __forceinline__ int s2(int k) { return (k + 8) & 1; }
__device__ __forceinline__ int s3(int k) { return (k + 9) % 3; }
__device__ __forceinline__ int s4(int k) { return (k + 8) & 3; }
__device__ __forceinline__ int s5(int k) { return (k + 10) % 5; }
__device__ __forceinline__ int s6(int k) { return (k + 12) % 6; }

// asynchronous global -> shared copy of one element (cp.async, L1-allocating)
template <typename T>
__device__ __forceinline__ void acopy(T *dst, const T *src) {
  unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  if (sizeof(T) == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}
// asynchronous global -> shared copy of 16 bytes (both addresses 16-byte
// aligned), cached in L2 only: the staged planes are not read again through
// L1, which is left to the per-level and per-column values
template <typename T>
__device__ __forceinline__ void acopy16(T *dst, const T *src) {
  unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void acommit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void await_groups() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// blocks per SM the register budget is sized for: FP32 tiles of 256 threads
// run two per SM (128 registers), everything else one
template <typename T, int TYv>
struct FullOcc {
  static constexpr int MINB = (sizeof(T) == 4 && TILE_X * TYv <= 256) ? 2 : 1;
};

template <typename T, int TYv>
__global__ void __launch_bounds__(TILE_X * TYv, FullOcc<T, TYv>::MINB) k_full(const DomDev *__restrict__ doms,
                                                        const WorkItem *__restrict__ items, int rO, int rC,
                                                        int rN, int rF, int first, const Eos E,
                                                        unsigned *__restrict__ watch) {
  using A = Ar<T>;
  using C = FullCfg<T, TYv>;
  constexpr int TX = C::TX, NT = C::NT, HX = C::HX, PL = C::PL, NLP = C::NLP;
  extern __shared__ __align__(16) unsigned char smraw[];
  FullSmem<T, PL> &S = *reinterpret_cast<FullSmem<T, PL> *>(smraw);
  const WorkItem W = items[blockIdx.x];
  const DomDev &D = doms[W.dom];
  const T dt2 = (T)(first ? D.dt : 2.0 * D.dt);
  const T nu = (T)(first ? 0.0 : D.ra_nu);
  const int tid = threadIdx.x;
  const int nx = D.nx, ny = D.ny, nz = D.nz, px = D.px;
  const long long plane = D.plane;
  const T *__restrict__ rpC = (const T *)D.f[rC][0];
  const T *__restrict__ ppC = (const T *)D.f[rC][1];
  const T *__restrict__ mC0 = (const T *)D.f[rC][2];
  const T *__restrict__ mC1 = (const T *)D.f[rC][3];
  const T *__restrict__ mC2 = (const T *)D.f[rC][4];
  const T *__restrict__ rpO = (const T *)D.f[rO][0];
  const T *__restrict__ ppO = (const T *)D.f[rO][1];
  const T *__restrict__ mO0 = (const T *)D.f[rO][2];
  const T *__restrict__ mO1 = (const T *)D.f[rO][3];
  const T *__restrict__ mO2 = (const T *)D.f[rO][4];
  const T *__restrict__ rhob = (const T *)D.rhob;
  const T *__restrict__ pb = (const T *)D.pb;
  const T *__restrict__ ipb = (const T *)D.ipb;
  const T *__restrict__ thb = (const T *)D.thb;
  const T *__restrict__ pik = (const T *)D.pik;
  const T *__restrict__ rhobc = (const T *)D.rhobc;
  const T *__restrict__ tau = (const T *)D.tau;
  const int i0 = W.i0, j0 = W.j0, k0 = W.k0, k1 = W.k1;

  // per-thread plane points of the haloed tile and their in-plane offsets
  // (periodic domains wrap the lateral coordinates; a refined box reads its
  // ghost frame, clamped to the padding where no computed point needs it)
  auto col_x = [&](int gi) { return D.periodic ? wrapi(gi, nx) : min(max(gi, -GX), px - GX - 1); };
  auto row_y = [&](int gj) { return D.periodic ? wrapi(gj, ny) : min(max(gj, -GH), D.py - GH - 1); };
  int loff[NLP], lpt[NLP], kbv[NLP];
#pragma unroll
  for (int s = 0; s < NLP; s++) {
    int p = tid + s * NT;
    lpt[s] = p;
    int hx = p % HX, hy = p / HX;
    loff[s] = (row_y(j0 - 2 + hy) + GH) * px + (col_x(i0 - 2 + hx) + GX);
    kbv[s] = p < PL ? D.kb[loff[s]] : KB_NONE;
  }
  // 16-byte chunks of the haloed rows (i0 is a multiple of 4, so a row of the
  // tile starts on a 16-byte boundary): this thread copies chunks tid,
  // tid + NT, .. of each field, whole where a chunk lies inside the row,
  // element by element (wrapped or clamped) where it crosses the periodic
  // seam or the end of the padding
  constexpr int VEC = 16 / sizeof(T), CPR = HX / VEC, NCH = CPR * C::HY, NCQ = (NCH + NT - 1) / NT;
  static_assert(HX % VEC == 0, "halo rows are whole chunks");
  int ch_dst[NCQ], ch_e[NCQ][VEC];  // destination, and source offsets of the elements
  bool ch_whole[NCQ];
#pragma unroll
  for (int q = 0; q < NCQ; q++) {
    const int t = tid + q * NT;
    const int row = t / CPR, col = t % CPR;
    const int x = i0 - 2 + VEC * col;
    const int rowoff = (row_y(j0 - 2 + row) + GH) * px;
    ch_dst[q] = t < NCH ? row * HX + VEC * col : -1;
    ch_whole[q] = D.periodic ? (x >= 0 && x + VEC <= nx) : (x >= -GX && x + VEC <= px - GX);
#pragma unroll
    for (int e = 0; e < VEC; e++) ch_e[q][e] = rowoff + col_x(x + e) + GX;
  }
  const T *__restrict__ ubC = (const T *)D.ub[rC];
  const int kmaxp = D.pz - GH - 1;  // highest plane inside the padding
  auto chunk = [&](T *dst, const T *src) {
#pragma unroll
    for (int q = 0; q < NCQ; q++) {
      if (ch_dst[q] < 0) continue;
      if (ch_whole[q]) {
        acopy16(dst + ch_dst[q], src + ch_e[q][0]);
      } else {
#pragma unroll
        for (int e = 0; e < VEC; e++) acopy(dst + ch_dst[q] + e, src + ch_e[q][e]);
      }
    }
  };
  // asynchronous copies of the raw fields of plane kk: the current-level
  // momentum when with_m (its ring has four slots), the n-1 fields when with_o
  auto issue = [&](int kk, bool with_m, bool with_o) {
    const long long zo = (long long)(min(kk, kmaxp) + GH) * plane;  // planes past the top are never used
    const int a5 = s5(kk), a4 = s4(kk);
    chunk(S.cr[a5], rpC + zo);
    chunk(S.cp[a5], ppC + zo);
    if (with_m) {
      chunk(S.cm[a4][0], mC0 + zo);
      chunk(S.cm[a4][1], mC1 + zo);
      chunk(S.cm[a4][2], mC2 + zo);
    }
    if (with_o) {
      chunk(S.op[a4], ppO + zo);
      chunk(S.om[a4][0], mO0 + zo);
      chunk(S.om[a4][1], mO1 + zo);
      chunk(S.om[a4][2], mO2 + zo);
    }
  };
  // totals of plane kk from its raw plane
  auto derive_e = [&](int kk, const T rb, const EosK<T> ek) {
    const int a5 = s5(kk), a4 = s4(kk);
#pragma unroll
    for (int s = 0; s < NLP; s++) {
      const int p = lpt[s];
      if (p < PL) {
        S.rh[a4][p] = A::add(rb, S.cr[a5][p]);
        S.th[a4][p] = ek.tot(E, S.cp[a5][p]);
      }
    }
  };
  auto derive = [&](int kk) {
    EosK<T> ek;
    ek.load(thb, pb, ipb, pik, kk + GH);
    derive_e(kk, rhob[kk + GH], ek);
  };
  // corner velocity of plane K = momentum / mean density of the 8 cells
  // around; corners at or below the terrain take the boundary-point velocity
  // of their column
  auto velocity = [&](int K) {
    const int sl = s4(K - 1), sh = s4(K), su = s3(K), sm = s4(K);
#pragma unroll
    for (int s = 0; s < NLP; s++) {
      const int p = lpt[s];
      const int hx = p % HX, hy = p / HX;
      if (p < PL && hx != 0 && hy != 0) {
        if (K <= kbv[s]) {
          const T *u = ubC + 3 * loff[s];
          S.uu[su][0][p] = u[0];
          S.uu[su][1][p] = u[1];
          S.uu[su][2][p] = u[2];
        } else {
          const T *lo = S.rh[sl], *hi = S.rh[sh];
          const int q00 = p - HX - 1, q01 = p - HX, q10 = p - 1, q11 = p;
          T iv = rinv(rho8(lo[q00], lo[q01], lo[q10], lo[q11], hi[q00], hi[q01], hi[q10], hi[q11]));
          S.uu[su][0][p] = S.cm[sm][0][p] * iv;
          S.uu[su][1][p] = S.cm[sm][1][p] * iv;
          S.uu[su][2][p] = S.cm[sm][2][p] * iv;
        }
      }
    }
  };
  // (rho theta)' at n-1 of plane kk (in-plane diffusion stencil)
  auto derive_old_e = [&](int kk, const EosK<T> ek) {
    const int a4 = s4(kk);
#pragma unroll
    for (int s = 0; s < NLP; s++) {
      const int p = lpt[s];
      if (p < PL) S.to[p] = ek.pert(E, S.op[a4][p]);
    }
  };

  const int tx = tid % TX, ty = tid / TX;
  const int i = i0 + tx, j = j0 + ty;
  const bool active = i >= D.ci0 && i < D.ci1 && j < D.cj1;
  // corners of a refined box outside -1 .. n+1 are ghost values from the coarser level
  const bool corner_active = active && i >= D.qi0 && j >= D.qj0;
  const int c = (ty + 2) * HX + (tx + 2);
  const long long own = active ? (long long)(j + GH) * px + (i + GX) : 0;
  const T qdx = (T)(0.25 / D.dx), qdy = (T)(0.25 / D.dy), qdz = (T)(0.25 / D.dz);  // 1/4 of the pressure-gradient quotient
  const T Sx = (T)(D.dy * D.dz), Sy = (T)(D.dx * D.dz), Sz = (T)(D.dx * D.dy);
  const T hSx = (T)(0.25 * D.dy * D.dz), hSy = (T)(0.25 * D.dx * D.dz), hSz = (T)(0.25 * D.dx * D.dy);
  const T v0inv = (T)(1.0 / (D.dx * D.dy * D.dz));
  const T kdif = (T)D.kdif, Cp = (T)D.Cp, g = (T)D.g, U = (T)D.U;
  const int kug = active ? D.kug[qidx(D, i, j)] : 0;
  // levels of this column whose cell and corner take the fourth-order
  // diffusion on every axis; the others take the wall-aware form
  const int dlo = active ? D.dcol[own].lo : 0, dhi = active ? D.dcol[own].hi : 0;

  // own column at n-1 for the vertical diffusion stencils, levels k-2 .. k+2
  T treg[5], mreg[5][3];
  auto own_old_e = [&](int a, int kk, const EosK<T> ek) {
    const int a4 = s4(kk);
    treg[a] = ek.pert(E, S.op[a4][c]);
    mreg[a][0] = S.om[a4][0][c];
    mreg[a][1] = S.om[a4][1][c];
    mreg[a][2] = S.om[a4][2][c];
  };
  auto own_old = [&](int a, int kk) {
    EosK<T> ek;
    ek.load(thb, pb, ipb, pik, kk + GH);
    own_old_e(a, kk, ek);
  };

  // prologue: raw planes k0-2 .. k0+2 (momentum from k0-1, n-1 fields from
  // k0-1: their rings have four slots), totals k0-2 .. k0+1, velocities
  // k0-1, k0; the own column at n-1 of plane k0-2 straight from memory
  for (int kk = k0 - 2; kk <= k0 + 2; kk++) issue(kk, kk != k0 - 2, kk != k0 - 2);
  acommit();
  {
    const long long o2 = (long long)(k0 - 2 + GH) * plane + own;
    EosK<T> ek;
    ek.load(thb, pb, ipb, pik, k0 - 2 + GH);
    treg[0] = ek.pert(E, ppO[o2]);
    mreg[0][0] = mO0[o2];
    mreg[0][1] = mO1[o2];
    mreg[0][2] = mO2[o2];
  }
  await_groups<0>();
  __syncthreads();
  for (int kk = k0 - 2; kk <= k0 + 1; kk++) derive(kk);
#pragma unroll
  for (int a = 1; a < 4; a++) own_old(a, k0 - 2 + a);
  __syncthreads();
  velocity(k0 - 1);
  velocity(k0);

  T fz_carry = 0, hz_carry = 0;  // high z-face fluxes of the previous plane
  // step watchdog: a non-finite value written, or the advective Courant
  // number sum_d |u_d| dt / d_d of a corner above 1 (the stability limit of
  // centred leapfrog advection)
  unsigned wflag = 0;
  const T cfx = (T)(D.dt / D.dx), cfy = (T)(D.dt / D.dy), cfz = (T)(D.dt / D.dz);
  for (int k = k0; k < k1; k++) {
    // phase 1: wait for plane k+2; once every thread is past the previous
    // plane (the barrier), the ring slots it read last are free and the
    // copies of plane k+3 go in flight; then the totals of plane k+2, the
    // velocities of plane k+1 and the n-1 fields of plane k
    T rO_ = 0;
    const long long o = (long long)(k + GH) * plane + own;
    if (active) rO_ = rpO[o];
    // base state of the levels this plane uses, loaded before the wait so
    // that their latency hides behind it
    EosK<T> ek0, ek2;
    ek0.load(thb, pb, ipb, pik, k + GH);
    ek2.load(thb, pb, ipb, pik, k + 2 + GH);
    const T rb2 = rhob[k + 2 + GH], tk = tau[k + GH];
    const T rbc[5] = {rhobc[k + GH - 2] * U, rhobc[k + GH - 1] * U, rhobc[k + GH] * U, rhobc[k + GH + 1] * U,
                      rhobc[k + GH + 2] * U};
    await_groups<0>();
    __syncthreads();
    issue(k + 3, true, true);
    acommit();
    derive_e(k + 2, rb2, ek2);
    velocity(k + 1);
    derive_old_e(k, ek0);
    own_old_e(4, k + 2, ek2);
    __syncthreads();
    // phase 2: the cell and corner of this thread on plane k
    if (active) {
      const int sk = s4(k), skm = s4(k - 1), skp = s4(k + 1);
      const int ck = s5(k), ckm = s5(k - 1);
      const T *R0 = S.rh[sk], *Rm = S.rh[skm], *Rp = S.rh[skp];
      const T *H0 = S.th[sk], *Hm = S.th[skm], *Hp = S.th[skp];
      const int uk = s3(k), ukp = s3(k + 1), ukm = s3(k - 1);
      const T *ux0 = S.uu[uk][0], *uy0 = S.uu[uk][1], *uz0 = S.uu[uk][2];
      const T *uxp = S.uu[ukp][0], *uyp = S.uu[ukp][1], *uzp = S.uu[ukp][2];
      // ---- scalar cell (i,j,k): face fluxes, lower-index cell first
      T fxm = face_flux(R0[c - 1], R0[c], ux0[c], ux0[c + HX], uxp[c], uxp[c + HX], Sx);
      T fxp = face_flux(R0[c], R0[c + 1], ux0[c + 1], ux0[c + 1 + HX], uxp[c + 1], uxp[c + 1 + HX], Sx);
      T fym = face_flux(R0[c - HX], R0[c], uy0[c], uy0[c + 1], uyp[c], uyp[c + 1], Sy);
      T fyp = face_flux(R0[c], R0[c + HX], uy0[c + HX], uy0[c + HX + 1], uyp[c + HX], uyp[c + HX + 1], Sy);
      // the low z-face of this cell is the high z-face of the cell below,
      // computed on the previous plane from the same values (same bits)
      T fzm = k > k0 ? fz_carry : face_flux(Rm[c], R0[c], uz0[c], uz0[c + 1], uz0[c + HX], uz0[c + HX + 1], Sz);
      T fzp = face_flux(R0[c], Rp[c], uzp[c], uzp[c + 1], uzp[c + HX], uzp[c + HX + 1], Sz);
      T hxm = face_flux(H0[c - 1], H0[c], ux0[c], ux0[c + HX], uxp[c], uxp[c + HX], Sx);
      T hxp = face_flux(H0[c], H0[c + 1], ux0[c + 1], ux0[c + 1 + HX], uxp[c + 1], uxp[c + 1 + HX], Sx);
      T hym = face_flux(H0[c - HX], H0[c], uy0[c], uy0[c + 1], uyp[c], uyp[c + 1], Sy);
      T hyp = face_flux(H0[c], H0[c + HX], uy0[c + HX], uy0[c + HX + 1], uyp[c + HX], uyp[c + HX + 1], Sy);
      T hzm = k > k0 ? hz_carry : face_flux(Hm[c], H0[c], uz0[c], uz0[c + 1], uz0[c + HX], uz0[c + HX + 1], Sz);
      T hzp = face_flux(H0[c], Hp[c], uzp[c], uzp[c + 1], uzp[c + HX], uzp[c + HX + 1], Sz);
      fz_carry = fzp;
      hz_carry = hzp;
      if (k == 0) { fzm = 0; hzm = 0; }                  // floor
      if (D.lid && k == nz - 1) { fzp = 0; hzp = 0; }    // rigid lid
      T RM = A::add(A::add(A::sub(fxp, fxm), A::sub(fyp, fym)), A::sub(fzp, fzm));
      T RH = A::add(A::add(A::sub(hxp, hxm), A::sub(hyp, hym)), A::sub(hzp, hzm));
      // artificial diffusion at n-1 of (rho theta)' and of the momentum
      // departure from the reference (rho_bar U, 0, 0): fourth order inside
      // the column's band, the wall-aware form next to the terrain and the lid
      const T *Tk = S.to;
      const int ok4 = s4(k);
      const bool wall = k < dlo || k >= dhi;
      T dd, dmv[3];
      if (!wall) {
        dd = d4(Tk[c - 2], Tk[c - 1], Tk[c], Tk[c + 1], Tk[c + 2]) +
             d4(Tk[c - 2 * HX], Tk[c - HX], Tk[c], Tk[c + HX], Tk[c + 2 * HX]) +
             d4(treg[0], treg[1], treg[2], treg[3], treg[4]);
#pragma unroll
        for (int d = 0; d < 3; d++) {
          const T *Mk = S.om[ok4][d];
          const T ref0 = d == 0 ? rbc[2] : T(0);
          T dm = d4(Mk[c - 2] - ref0, Mk[c - 1] - ref0, Mk[c] - ref0, Mk[c + 1] - ref0, Mk[c + 2] - ref0) +
                 d4(Mk[c - 2 * HX] - ref0, Mk[c - HX] - ref0, Mk[c] - ref0, Mk[c + HX] - ref0,
                    Mk[c + 2 * HX] - ref0);
          if (d == 0)
            dm += d4(mreg[0][0] - rbc[0], mreg[1][0] - rbc[1], mreg[2][0] - ref0, mreg[3][0] - rbc[3],
                     mreg[4][0] - rbc[4]);
          else
            dm += d4(mreg[0][d], mreg[1][d], mreg[2][d], mreg[3][d], mreg[4][d]);
          dmv[d] = dm;
        }
      } else {
        const DiffCol &Q = D.dcol[own];
        const int ct = Q.ctop, vt = Q.vtop;
        dd = diff_axis(Tk[c - 2], Tk[c - 1], Tk[c], Tk[c + 1], Tk[c + 2], fluid_at(k, Q.cx[0], ct),
                       fluid_at(k, Q.cx[1], ct), fluid_at(k, Q.cx[2], ct), fluid_at(k, Q.cx[3], ct), true) +
             diff_axis(Tk[c - 2 * HX], Tk[c - HX], Tk[c], Tk[c + HX], Tk[c + 2 * HX], fluid_at(k, Q.cy[0], ct),
                       fluid_at(k, Q.cy[1], ct), fluid_at(k, Q.cy[2], ct), fluid_at(k, Q.cy[3], ct), true) +
             diff_axis(treg[0], treg[1], treg[2], treg[3], treg[4], fluid_at(k - 2, Q.c0, ct),
                       fluid_at(k - 1, Q.c0, ct), fluid_at(k + 1, Q.c0, ct), fluid_at(k + 2, Q.c0, ct), true);
        const bool fx0 = fluid_at(k, Q.vx[0], vt), fx1 = fluid_at(k, Q.vx[1], vt), fx2 = fluid_at(k, Q.vx[2], vt),
                   fx3 = fluid_at(k, Q.vx[3], vt);
        const bool fy0 = fluid_at(k, Q.vy[0], vt), fy1 = fluid_at(k, Q.vy[1], vt), fy2 = fluid_at(k, Q.vy[2], vt),
                   fy3 = fluid_at(k, Q.vy[3], vt);
        const bool fz0 = fluid_at(k - 2, Q.v0, vt), fz1 = fluid_at(k - 1, Q.v0, vt),
                   fz2 = fluid_at(k + 1, Q.v0, vt), fz3 = fluid_at(k + 2, Q.v0, vt);
#pragma unroll
        for (int d = 0; d < 3; d++) {
          const T *Mk = S.om[ok4][d];
          const T ref0 = d == 0 ? rbc[2] : T(0);
          T dm = diff_axis(Mk[c - 2] - ref0, Mk[c - 1] - ref0, Mk[c] - ref0, Mk[c + 1] - ref0, Mk[c + 2] - ref0,
                           fx0, fx1, fx2, fx3, false) +
                 diff_axis(Mk[c - 2 * HX] - ref0, Mk[c - HX] - ref0, Mk[c] - ref0, Mk[c + HX] - ref0,
                           Mk[c + 2 * HX] - ref0, fy0, fy1, fy2, fy3, false);
          if (d == 0)
            dm += diff_axis(mreg[0][0] - rbc[0], mreg[1][0] - rbc[1], mreg[2][0] - ref0, mreg[3][0] - rbc[3],
                            mreg[4][0] - rbc[4], fz0, fz1, fz2, fz3, false);
          else
            dm += diff_axis(mreg[0][d], mreg[1][d], mreg[2][d], mreg[3][d], mreg[4][d], fz0, fz1, fz2, fz3, false);
          dmv[d] = dm;
        }
      }
      T Dth = -kdif * dd;
      const EosK<T> &ek = ek0;
      T rC_ = S.cr[ck][c], pC_ = S.cp[ck][c];
      const T mcur[3] = {S.cm[sk][0][c], S.cm[sk][1][c], S.cm[sk][2][c]};
      T pO_ = S.op[s4(k)][c];
      T rN_ = rO_ - dt2 * (RM * v0inv);
      T pN_ = pO_ - dt2 * Cp * ek.exner(E, pC_) * (RH * v0inv - Dth);
      if (k < kug) { rN_ = 0; pN_ = 0; }
      T rF_ = rC_ + nu * (rN_ - T(2) * rC_ + rO_);
      T pF_ = pC_ + nu * (pN_ - T(2) * pC_ + pO_);
      if (k < kug) { rF_ = 0; pF_ = 0; }

      // ---- velocity cell centred on corner (i,j,K=k): Eqs. momentum_u_d .. w_d
      // face densities and pressures of the velocity cell: means over the 4
      // cells touching each face, from the vertical pair sums of the 4
      // cell columns around the corner
      const int cW = c - 1, cS = c - HX, cSW = c - HX - 1;
      const T v00 = Rm[cSW] + R0[cSW], v10 = Rm[cS] + R0[cS], v01 = Rm[cW] + R0[cW], v11 = Rm[c] + R0[c];
      const T rE = (v10 + v11) * T(0.25), rW = (v00 + v01) * T(0.25);
      const T rNn = (v01 + v11) * T(0.25), rS = (v00 + v10) * T(0.25);
      const T rT = ((R0[cSW] + R0[cS]) + (R0[cW] + R0[c])) * T(0.25);
      const T rB = ((Rm[cSW] + Rm[cS]) + (Rm[cW] + Rm[c])) * T(0.25);
      const T *uxm = S.uu[ukm][0], *uym = S.uu[ukm][1], *uzm = S.uu[ukm][2];
      T u0[3] = {ux0[c], uy0[c], uz0[c]};
      T uE[3] = {ux0[c + 1], uy0[c + 1], uz0[c + 1]};
      T uW[3] = {ux0[c - 1], uy0[c - 1], uz0[c - 1]};
      T uN[3] = {ux0[c + HX], uy0[c + HX], uz0[c + HX]};
      T uS[3] = {ux0[c - HX], uy0[c - HX], uz0[c - HX]};
      T uT[3] = {uxp[c], uyp[c], uzp[c]};
      T uB[3] = {uxm[c], uym[c], uzm[c]};
      // half the mass flux through each face (face density x mean normal
      // velocity x area); the advected value is the mean of the two corners:
      // sum_f g_f (u0 + u_f) = u0 sum_f g_f + sum_f g_f u_f
      const T gE = rE * (u0[0] + uE[0]) * hSx, gW = rW * (uW[0] + u0[0]) * hSx;
      const T gN = rNn * (u0[1] + uN[1]) * hSy, gS = rS * (uS[1] + u0[1]) * hSy;
      const T gT = rT * (u0[2] + uT[2]) * hSz, gB = rB * (uB[2] + u0[2]) * hSz;
      const T gsum = ((gE - gW) + (gN - gS)) + (gT - gB);
      const T *P0 = S.cp[ck], *Pm = S.cp[ckm];
      const T w00 = Pm[cSW] + P0[cSW], w10 = Pm[cS] + P0[cS], w01 = Pm[cW] + P0[cW], w11 = Pm[c] + P0[c];
      const T pE = w10 + w11, pW = w00 + w01, pNn = w01 + w11, pS = w00 + w10;
      const T pT = (P0[cSW] + P0[cS]) + (P0[cW] + P0[c]);
      const T pB = (Pm[cSW] + Pm[cS]) + (Pm[cW] + Pm[c]);
      const T *Q0 = S.cr[ck], *Qm = S.cr[ckm];
      T r8 = (Q0[cSW] + Q0[cS] + Q0[cW] + Q0[c]) + (Qm[cSW] + Qm[cS] + Qm[cW] + Qm[c]);
      T pg[3] = {(pE - pW) * qdx, (pNn - pS) * qdy, (pT - pB) * qdz};
      T mnew[3], mflt[3];
#pragma unroll
      for (int d = 0; d < 3; d++) {
        T adv = u0[d] * gsum + (((gE * uE[d] - gW * uW[d]) + (gN * uN[d] - gS * uS[d])) + (gT * uT[d] - gB * uB[d]));
        T tend = -adv * v0inv - pg[d];
        if (d == 2) tend -= g * r8 * T(0.125);
        const T ref0 = d == 0 ? rbc[2] : T(0);
        T mold = mreg[2][d];
        tend += -kdif * dmv[d] - tk * (mold - ref0);
        mnew[d] = mold + dt2 * tend;
        mflt[d] = mcur[d] + nu * (mnew[d] - T(2) * mcur[d] + mold);
      }
      {
        const T chk = ((rN_ + pN_) + (mnew[0] + mnew[1])) + mnew[2];
        if (!isfinite(chk)) wflag |= WATCH_NONFINITE;
        if (fabs(u0[0]) * cfx + fabs(u0[1]) * cfy + fabs(u0[2]) * cfz > T(1)) wflag |= WATCH_COURANT;
      }
      // every store after every shared-memory read of the plane (a store
      // through a generic pointer would otherwise order the later reads)
      ((T *)D.f[rN][0])[o] = rN_;
      ((T *)D.f[rN][1])[o] = pN_;
      ((T *)D.f[rF][0])[o] = rF_;
      ((T *)D.f[rF][1])[o] = pF_;
      if (corner_active) {
#pragma unroll
        for (int d = 0; d < 3; d++) {
          ((T *)D.f[rN][2 + d])[o] = mnew[d];
          ((T *)D.f[rF][2 + d])[o] = mflt[d];
        }
      }
    }
#pragma unroll
    for (int a = 0; a < 4; a++) {
      treg[a] = treg[a + 1];
      mreg[a][0] = mreg[a + 1][0];
      mreg[a][1] = mreg[a + 1][1];
      mreg[a][2] = mreg[a + 1][2];
    }
  }
  await_groups<0>();
  wflag = __reduce_or_sync(0xffffffffu, wflag);
  if (wflag && (tid & 31) == 0 && watch) atomicOr(watch, wflag);
}

#include "pair.cuh"

// ------------------------------------------------------------------ cut cells and merge groups
template <typename T>
__device__ __forceinline__ T cell_rho(const DomDev &D, const T *rp, const T *rhob, int i, int j, int k) {
  return Ar<T>::add(rhob[k + GH], rp[widx(D, i, j, k)]);
}

// corner density (the same operations as the full-cell stencil)
template <typename T>
__device__ __forceinline__ T corner_rho(const DomDev &D, const T *rp, const T *rhob, int I, int J, int K) {
  return rho8(cell_rho(D, rp, rhob, I - 1, J - 1, K - 1), cell_rho(D, rp, rhob, I, J - 1, K - 1),
              cell_rho(D, rp, rhob, I - 1, J, K - 1), cell_rho(D, rp, rhob, I, J, K - 1),
              cell_rho(D, rp, rhob, I - 1, J - 1, K), cell_rho(D, rp, rhob, I, J - 1, K),
              cell_rho(D, rp, rhob, I - 1, J, K), cell_rho(D, rp, rhob, I, J, K));
}

// padded column of corner (I, J), wrapped on periodic domains
__device__ __forceinline__ long long wqidx(const DomDev &D, int I, int J) {
  return D.periodic ? qidx(D, wrapi(I, D.nx), wrapi(J, D.ny)) : qidx(D, I, J);
}

// corner velocity (the same operations as the full-cell stencil): the
// boundary-point velocity ub for corners at or below the terrain (when ub is
// given), else momentum / corner density
template <typename T>
__device__ __forceinline__ void corner_u(const DomDev &D, const T *rp, const T *const *M, const T *rhob,
                                         const T *ub, int I, int J, int K, T u[3]) {
  if (ub) {
    const long long q = wqidx(D, I, J);
    if (K <= D.kb[q]) {
      u[0] = ub[3 * q];
      u[1] = ub[3 * q + 1];
      u[2] = ub[3 * q + 2];
      return;
    }
  }
  T iv = rinv(corner_rho(D, rp, rhob, I, J, K));
  long long o = widx(D, I, J, K);
  u[0] = M[0][o] * iv;
  u[1] = M[1][o] * iv;
  u[2] = M[2][o] * iv;
}

// The diffusion sum S of a scalar cell (i, j, k) with the wall-aware axis
// terms, from the column descriptor Q and a function f(i, j, k) giving the
// diffused value at n-1.
template <typename T, typename F>
__device__ __forceinline__ T scalar_diffusion(const DiffCol &Q, int k, F &&f, int i, int j) {
  const int ct = Q.ctop;
  const T c = f(i, j, k);
  return diff_axis(f(i - 2, j, k), f(i - 1, j, k), c, f(i + 1, j, k), f(i + 2, j, k), fluid_at(k, Q.cx[0], ct),
                   fluid_at(k, Q.cx[1], ct), fluid_at(k, Q.cx[2], ct), fluid_at(k, Q.cx[3], ct), true) +
         diff_axis(f(i, j - 2, k), f(i, j - 1, k), c, f(i, j + 1, k), f(i, j + 2, k), fluid_at(k, Q.cy[0], ct),
                   fluid_at(k, Q.cy[1], ct), fluid_at(k, Q.cy[2], ct), fluid_at(k, Q.cy[3], ct), true) +
         diff_axis(f(i, j, k - 2), f(i, j, k - 1), c, f(i, j, k + 1), f(i, j, k + 2), fluid_at(k - 2, Q.c0, ct),
                   fluid_at(k - 1, Q.c0, ct), fluid_at(k + 1, Q.c0, ct), fluid_at(k + 2, Q.c0, ct), true);
}

template <typename T>
__global__ void k_groups(const DomDev *__restrict__ doms, const GroupRec *__restrict__ recs, int ng,
                         const int32_t *__restrict__ members, int rO, int rC, int rN, int rF, int first) {
  using A = Ar<T>;
  int gi = blockIdx.x * blockDim.x + threadIdx.x;
  if (gi >= ng) return;
  const GroupRec R = recs[gi];
  const DomDev &D = doms[R.dom];
  const T dt2 = (T)(first ? D.dt : 2.0 * D.dt);
  const T nu = (T)(first ? 0.0 : D.ra_nu);
  const int nx = D.nx, ny = D.ny, nz = D.nz;
  const T *rpC = (const T *)D.f[rC][0];
  const T *ppC = (const T *)D.f[rC][1];
  const T *MC[3] = {(const T *)D.f[rC][2], (const T *)D.f[rC][3], (const T *)D.f[rC][4]};
  const T *ubC = (const T *)D.ub[rC];
  const T *rpO = (const T *)D.f[rO][0];
  const T *ppO = (const T *)D.f[rO][1];
  const T *rhob = (const T *)D.rhob, *pb = (const T *)D.pb, *thb = (const T *)D.thb, *pik = (const T *)D.pik;
  const T *ipb = (const T *)D.ipb;
  const T Sfull[3] = {(T)(D.dy * D.dz), (T)(D.dx * D.dz), (T)(D.dx * D.dy)};
  T rm = 0, rh = 0;
  for (int a = 0; a < R.count; a++) {
    int m = members[R.start + a];
    int i = m % nx, j = (m / nx) % ny, k = m / (nx * ny);
    // the eight corner velocities of the cell, [dk][dj][di]
    T uc8[2][2][2][3];
#pragma unroll
    for (int dk = 0; dk < 2; dk++)
#pragma unroll
      for (int dj = 0; dj < 2; dj++)
#pragma unroll
        for (int di = 0; di < 2; di++) corner_u(D, rpC, MC, rhob, ubC, i + di, j + dj, k + dk, uc8[dk][dj][di]);
    const T phm = cell_rho(D, rpC, rhob, i, j, k);
    const T thm = theta_tot(D, thb, pb, ipb, k + GH, ppC[widx(D, i, j, k)]);
    for (int ax = 0; ax < 3; ax++)
      for (int sd = 0; sd <= 1; sd++) {
        int ni = i, nj = j, nk = k;
        double Ap;
        const T *uc[4];
        if (ax == 0) {
          int I = i + sd;
          ni = i + (sd ? 1 : -1);
          Ap = D.ax[cid(D, wrapi(I, nx), j, k)];
          uc[0] = uc8[0][0][sd]; uc[1] = uc8[0][1][sd]; uc[2] = uc8[1][0][sd]; uc[3] = uc8[1][1][sd];
        } else if (ax == 1) {
          int J = j + sd;
          nj = j + (sd ? 1 : -1);
          Ap = D.ay[cid(D, i, wrapi(J, ny), k)];
          uc[0] = uc8[0][sd][0]; uc[1] = uc8[0][sd][1]; uc[2] = uc8[1][sd][0]; uc[3] = uc8[1][sd][1];
        } else {
          int K = k + sd;
          nk = k + (sd ? 1 : -1);
          Ap = D.az[((long long)K * ny + j) * nx + i];
          uc[0] = uc8[sd][0][0]; uc[1] = uc8[sd][0][1]; uc[2] = uc8[sd][1][0]; uc[3] = uc8[sd][1][1];
        }
        if (Ap == 0.0) continue;
        if (nk < 0 || nk >= nz) continue;
        long long nb = cid(D, wrapi(ni, nx), wrapi(nj, ny), nk);
        if (D.cls[nb] != C_UG && D.root[nb] == R.host) continue;  // face inside the group
        T phn = cell_rho(D, rpC, rhob, ni, nj, nk);
        T thn = theta_tot(D, thb, pb, ipb, nk + GH, ppC[widx(D, ni, nj, nk)]);
        T S = (Ap == 1.0) ? Sfull[ax] : (T)(Ap * (double)Sfull[ax]);
        T fm, fh;
        if (sd) {
          fm = face_flux(phm, phn, uc[0][ax], uc[1][ax], uc[2][ax], uc[3][ax], S);
          fh = face_flux(thm, thn, uc[0][ax], uc[1][ax], uc[2][ax], uc[3][ax], S);
          rm = A::add(rm, fm);
          rh = A::add(rh, fh);
        } else {
          fm = face_flux(phn, phm, uc[0][ax], uc[1][ax], uc[2][ax], uc[3][ax], S);
          fh = face_flux(thn, thm, uc[0][ax], uc[1][ax], uc[2][ax], uc[3][ax], S);
          rm = A::sub(rm, fm);
          rh = A::sub(rh, fh);
        }
      }
  }
  // host update
  int h = R.host;
  int ih = h % nx, jh = (h / nx) % ny, kh = h / (nx * ny);
  auto tho = [&](int ii, int jj, int kk) { return theta_pert(D, thb, pb, ipb, kk + GH, ppO[widx(D, ii, jj, kk)]); };
  // wall-aware diffusion of (rho theta)' at n-1 at the host
  T dd = scalar_diffusion<T>(D.dcol[qidx(D, ih, jh)], kh, tho, ih, jh);
  T Dth = -(T)D.kdif * dd;
  long long oh = pidx(D, ih, jh, kh);
  T rC_ = rpC[oh], pC_ = ppC[oh], rO_ = rpO[oh], pO_ = ppO[oh];
  T VG = (T)R.vg;
  T rN_ = rO_ - dt2 * (rm / VG);
  T pN_ = pO_ - dt2 * (T)D.Cp * exner_fac(D, pik, pb, ipb, kh + GH, pC_) * (rh / VG - Dth);
  T rF_ = rC_ + nu * (rN_ - T(2) * rC_ + rO_);
  T pF_ = pC_ + nu * (pN_ - T(2) * pC_ + pO_);
  for (int a = 0; a < R.count; a++) {
    int m = members[R.start + a];
    int i = m % nx, j = (m / nx) % ny, k = m / (nx * ny);
    long long o = pidx(D, i, j, k);
    ((T *)D.f[rN][0])[o] = rN_;
    ((T *)D.f[rN][1])[o] = pN_;
    ((T *)D.f[rF][0])[o] = rF_;
    ((T *)D.f[rF][1])[o] = pF_;
  }
}

// ------------------------------------------------------------------ velocity diagnosis
template <typename T>
__global__ void k_diag(const DomDev *__restrict__ doms, const ColItem *__restrict__ cols, int ncols, int rV,
                       int rC, int rO, int rF, int first, int filter) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ncols) return;
  const ColItem CI = cols[t];
  const DomDev &D = doms[CI.dom];
  const T nu = (T)(first ? 0.0 : D.ra_nu);
  const int I = CI.I, J = CI.J;
  const T *rp = (const T *)D.f[rV][0];
  T *M[3] = {(T *)D.f[rV][2], (T *)D.f[rV][3], (T *)D.f[rV][4]};
  const T *const *Mc = (const T *const *)M;
  const T *rhob = (const T *)D.rhob;
  const long long q = qidx(D, I, J);
  // boundary point: bilinear in the nearest plane, then free-slip projection
  int K = D.bK[q], i0 = D.bI[q], j0 = D.bJ[q];
  T a = (T)D.ba[q], b = (T)D.bb[q];
  T w[4] = {(T(1) - a) * (T(1) - b), a * (T(1) - b), (T(1) - a) * b, a * b};
  int ci[4] = {i0, i0 + 1, i0, i0 + 1}, cj[4] = {j0, j0, j0 + 1, j0 + 1};
  T uN[3] = {0, 0, 0};
  for (int s = 0; s < 4; s++) {
    if (w[s] == T(0)) continue;
    T u[3];
    corner_u<T>(D, rp, Mc, rhob, nullptr, ci[s], cj[s], K, u);
    for (int d = 0; d < 3; d++) uN[d] += w[s] * u[d];
  }
  T n[3] = {(T)D.bn[3 * q], (T)D.bn[3 * q + 1], (T)D.bn[3 * q + 2]};
  T ub[3];
  if (D.bc_slip) {
    T un = uN[0] * n[0] + uN[1] * n[1] + uN[2] * n[2];
    for (int d = 0; d < 3; d++) ub[d] = uN[d] - un * n[d];
  } else {
    ub[0] = ub[1] = ub[2] = 0;
  }
  T *ubv = (T *)D.ub[rV];
  for (int d = 0; d < 3; d++) ubv[3 * q + d] = ub[d];
  const T *__restrict__ mcur[3] = {(const T *)D.f[rC][2], (const T *)D.f[rC][3], (const T *)D.f[rC][4]};
  const T *__restrict__ mold[3] = {(const T *)D.f[rO][2], (const T *)D.f[rO][3], (const T *)D.f[rO][4]};
  T *__restrict__ mflt[3] = {(T *)D.f[rF][2], (T *)D.f[rF][3], (T *)D.f[rF][4]};
  // the four cell columns around the corner column, in the order of the
  // corner density (i-1,j-1), (i,j-1), (i-1,j), (i,j); totals of cell level k
  // are carried from one corner level to the next
  const long long plane = D.plane;
  const long long oc[4] = {widx(D, I - 1, J - 1, -GH), widx(D, I, J - 1, -GH), widx(D, I - 1, J, -GH),
                           widx(D, I, J, -GH)};
  const long long own = pidx(D, I, J, -GH);
  auto level = [&](int k, T r[4]) {
    const T rb = rhob[k + GH];
    const long long z = (long long)(k + GH) * plane;
#pragma unroll
    for (int s = 0; s < 4; s++) r[s] = Ar<T>::add(rb, rp[oc[s] + z]);
  };
  auto store = [&](int KK, const T lo[4], const T hi[4], const T u[3]) {
    const long long o = own + (long long)(KK + GH) * plane;
    const T rc = rho8(lo[0], lo[1], lo[2], lo[3], hi[0], hi[1], hi[2], hi[3]);
#pragma unroll
    for (int d = 0; d < 3; d++) {
      T mv = rc * u[d];
      M[d][o] = mv;
      if (filter) {
        T mc = mcur[d][o];
        mflt[d][o] = mc + nu * (mv - T(2) * mc + mold[d][o]);
      }
    }
  };
  // corner levels from -GH+1: the density of corner K averages cell levels
  // K-1 and K, and the lowest padded cell level is -GH
  const int kt = D.ktop[q];
  T lo[4], hi[4];
  level(-GH, lo);
  for (int KK = -GH + 1; KK <= kt; KK++) {
    level(KK, hi);
    const long long p = own + (long long)(KK + GH) * plane;
    const int8_t v = D.vcls[p];
    if (v != V_PRED) {
      T u[3];
      if (v == V_UG) {
        u[0] = ub[0]; u[1] = ub[1]; u[2] = ub[2];
      } else {
        int ka = D.mK[p];
        T gm = (T)D.mg[p];
        T ua[3];
        corner_u<T>(D, rp, Mc, rhob, nullptr, I, J, ka, ua);
        for (int d = 0; d < 3; d++) u[d] = gm * ua[d] + (T(1) - gm) * ub[d];
      }
      store(KK, lo, hi, u);
    }
#pragma unroll
    for (int s = 0; s < 4; s++) lo[s] = hi[s];
  }
  if (D.lid) {
    T ul[3];
    corner_u<T>(D, rp, Mc, rhob, nullptr, I, J, D.nz - 1, ul);
    ul[2] = 0;
    level(D.nz - 1, lo);
    for (int KK = D.nz; KK < D.nz + GH; KK++) {
      level(KK, hi);
      store(KK, lo, hi, ul);
#pragma unroll
      for (int s = 0; s < 4; s++) lo[s] = hi[s];
    }
  }
}

// initial momentum rho_corner * U on the predicted points of level r
template <typename T>
__global__ void k_init_momentum(const DomDev *__restrict__ dom, int r, double U) {
  const DomDev &D = *dom;
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int wx = D.ci1 - D.qi0, wy = D.cj1 - D.qj0;
  long long n = (long long)wx * wy * D.ck1;
  if (t >= n) return;
  int I = (int)(t % wx) + D.qi0, J = (int)((t / wx) % wy) + D.qj0, K = (int)(t / ((long long)wx * wy));
  long long o = pidx(D, I, J, K);
  if (D.vcls[o] != V_PRED) return;
  const T *rp = (const T *)D.f[r][0];
  T rc = corner_rho(D, rp, (const T *)D.rhob, I, J, K);
  ((T *)D.f[r][2])[o] = rc * (T)U;
}

// ------------------------------------------------------------------ diagnostics
// Compensated sums and maxima (Sec 2.2: the mass the scheme conserves):
// Neumaier per thread over a fixed grid-stride share of the cells, then
// warp-shuffle TwoSum trees within each block and over the block partials.
// Fixed block count and fixed order, so the result does not depend on
// scheduling and repeats bit for bit.
constexpr int DIAG_BLOCKS = 256, DIAG_TPB = 256;

template <typename T>
__global__ void k_diag_partial(const DomDev *__restrict__ dom, int r, double *part) {
  const DomDev &D = *dom;
  const T *rp = (const T *)D.f[r][0];
  const T *pp = (const T *)D.f[r][1];
  const T *M[3] = {(const T *)D.f[r][2], (const T *)D.f[r][3], (const T *)D.f[r][4]};
  const T *rhob = (const T *)D.rhob;
  const double V0 = D.dx * D.dy * D.dz;
  long long n = (long long)D.nx * D.ny * D.nz;
  NSum<T> acc{0, 0};
  double mu = 0, mw = 0, bad = 0;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    int i = (int)(t % D.nx), j = (int)((t / D.nx) % D.ny), k = (int)(t / ((long long)D.nx * D.ny));
    long long o = pidx(D, i, j, k);
    T rv = rp[o];
    acc.add((T)(D.vf[t] * V0) * rv);
    T vals[5] = {rv, pp[o], M[0][o], M[1][o], M[2][o]};
    for (int a = 0; a < 5; a++)
      if (!isfinite((double)vals[a])) bad += 1;
    if (D.vcls[o] == V_PRED) {
      T rc = corner_rho(D, rp, rhob, i, j, k);
      double uu = fabs((double)(M[0][o] / rc)), ww = fabs((double)(M[2][o] / rc));
      mu = fmax(mu, uu);
      mw = fmax(mw, ww);
    }
  }
  __shared__ CSum shc[DIAG_TPB / 32];
  __shared__ double shm[DIAG_TPB / 32];
  const CSum m = block_csum<DIAG_TPB>(CSum{(double)acc.s, (double)acc.c}, shc);
  const CSum nb = block_csum<DIAG_TPB>(CSum{bad, 0.0}, shc);
  const double a2 = block_max<DIAG_TPB>(mu, shm), a3 = block_max<DIAG_TPB>(mw, shm);
  if (threadIdx.x == 0) {
    part[5 * blockIdx.x + 0] = m.s;
    part[5 * blockIdx.x + 1] = m.c;
    part[5 * blockIdx.x + 2] = a2;
    part[5 * blockIdx.x + 3] = a3;
    part[5 * blockIdx.x + 4] = nb.s;
  }
}

// One block of DIAG_TPB threads over the nb block partials (thread t takes
// partials t, t + DIAG_TPB, ..), then the same trees.
__global__ void k_diag_final(const double *part, int nb, double *out) {
  CSum m{0.0, 0.0}, bad{0.0, 0.0};
  double a2 = 0, a3 = 0;
  for (int b = threadIdx.x; b < nb; b += DIAG_TPB) {
    m = csum_add(m, CSum{part[5 * b], part[5 * b + 1]});
    a2 = fmax(a2, part[5 * b + 2]);
    a3 = fmax(a3, part[5 * b + 3]);
    bad = csum_add(bad, CSum{part[5 * b + 4], 0.0});
  }
  __shared__ CSum shc[DIAG_TPB / 32];
  __shared__ double shm[DIAG_TPB / 32];
  m = block_csum<DIAG_TPB>(m, shc);
  bad = block_csum<DIAG_TPB>(bad, shc);
  a2 = block_max<DIAG_TPB>(a2, shm);
  a3 = block_max<DIAG_TPB>(a3, shm);
  if (threadIdx.x == 0) {
    out[0] = m.s + m.c;
    out[1] = m.c;
    out[2] = a2;
    out[3] = a3;
    out[4] = bad.s;
  }
}


// ------------------------------------------------------------------ derived output (not on the step path)
// Corner velocity for corners K = 0 .. nz (the velocity every flux uses:
// the boundary-point value at or below the terrain, else momentum / corner
// density) or, for which == 3, the potential-temperature perturbation of each
// cell, theta' = ((rho theta)' - theta_bar rho') / (rho_bar + rho') with
// theta_bar = (rho theta)_bar / rho_bar; FP64 host layout.
template <typename T>
__global__ void k_derived(const DomDev *__restrict__ dom, int r, int which, double *__restrict__ out) {
  const DomDev &D = *dom;
  const long long ncol = (long long)D.nx * D.ny;
  const long long n = ncol * (which == 3 ? D.nz : D.nz + 1);
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const int i = (int)(t % D.nx), j = (int)((t / D.nx) % D.ny), k = (int)(t / ncol);
  const T *rp = (const T *)D.f[r][0];
  const T *rhob = (const T *)D.rhob;
  if (which == 3) {
    const long long o = pidx(D, i, j, k);
    const int kp = k + GH;
    const T *thb = (const T *)D.thb;
    const double X = (double)theta_pert(D, thb, (const T *)D.pb, (const T *)D.ipb, kp, ((const T *)D.f[r][1])[o]);
    const double rb = (double)rhob[kp], rv = (double)rp[o];
    out[t] = (X - (double)thb[kp] / rb * rv) / (rb + rv);
    return;
  }
  const T *M[3] = {(const T *)D.f[r][2], (const T *)D.f[r][3], (const T *)D.f[r][4]};
  T u[3];
  corner_u<T>(D, rp, M, rhob, (const T *)D.ub[r], i, j, k, u);
  out[t] = (double)u[which];
}

// Heat content sum_G V_G (rho theta)'_G: every member cell of a merge group
// adds its volume times the host's (rho theta)' (evaluated at the host's
// level); cells below the terrain have no volume.  Neumaier sums in FP64,
// fixed block count and order.
template <typename T>
__global__ void k_heat_partial(const DomDev *__restrict__ dom, int r, double *part) {
  const DomDev &D = *dom;
  const T *pp = (const T *)D.f[r][1];
  const double V0 = D.dx * D.dy * D.dz;
  const long long ncol = (long long)D.nx * D.ny, n = ncol * D.nz;
  NSum<double> acc{0, 0};
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const int32_t h = D.root[t];
    if (h < 0 || D.vf[t] == 0.0) continue;
    const int ih = (int)(h % D.nx), jh = (int)((h / D.nx) % D.ny), kh = (int)(h / ncol);
    const T x = theta_pert(D, (const T *)D.thb, (const T *)D.pb, (const T *)D.ipb, kh + GH, pp[pidx(D, ih, jh, kh)]);
    acc.add(D.vf[t] * V0 * (double)x);
  }
  __shared__ CSum shc[DIAG_TPB / 32];
  const CSum h = block_csum<DIAG_TPB>(CSum{acc.s, acc.c}, shc);
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = h.s;
    part[2 * blockIdx.x + 1] = h.c;
  }
}

__global__ void k_heat_final(const double *part, int nb, double *out) {
  CSum h{0.0, 0.0};
  for (int b = threadIdx.x; b < nb; b += DIAG_TPB) h = csum_add(h, CSum{part[2 * b], part[2 * b + 1]});
  __shared__ CSum shc[DIAG_TPB / 32];
  h = block_csum<DIAG_TPB>(h, shc);
  if (threadIdx.x == 0) {
    out[0] = h.s + h.c;
    out[1] = h.c;
  }
}

// Global error norms (appendix accuracy test): the corner velocity component
// `which` of model A against the finer model B at the corners the grids
// share (spacing ratio p/q: corner q I' of A is corner p I' of B), over the
// shared corners with K >= kmin of A; Neumaier sums of |d| and d^2 in FP64,
// fixed block count and order.
template <typename TA, typename TB>
__global__ void k_norms(const DomDev *__restrict__ A, int ra, const DomDev *__restrict__ B, int rb, int which, int p,
                        int q, int kmin, double *part) {
  const DomDev &Da = *A, &Db = *B;
  const int mx = (Da.nx + q - 1) / q, my = (Da.ny + q - 1) / q, k0 = (kmin + q - 1) / q;
  const long long ncol = (long long)mx * my, n = ncol * (Da.nz / q + 1 - k0);
  const TA *Ma[3] = {(const TA *)Da.f[ra][2], (const TA *)Da.f[ra][3], (const TA *)Da.f[ra][4]};
  const TB *Mb[3] = {(const TB *)Db.f[rb][2], (const TB *)Db.f[rb][3], (const TB *)Db.f[rb][4]};
  NSum<double> s1{0, 0}, s2{0, 0};
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const int Ip = (int)(t % mx), Jp = (int)((t / mx) % my), Kp = k0 + (int)(t / ncol);
    TA ua[3];
    TB ub[3];
    corner_u<TA>(Da, (const TA *)Da.f[ra][0], Ma, (const TA *)Da.rhob, (const TA *)Da.ub[ra], q * Ip, q * Jp, q * Kp,
                 ua);
    corner_u<TB>(Db, (const TB *)Db.f[rb][0], Mb, (const TB *)Db.rhob, (const TB *)Db.ub[rb], p * Ip, p * Jp, p * Kp,
                 ub);
    const double d = (double)ua[which] - (double)ub[which];
    s1.add(fabs(d));
    s2.add(d * d);
  }
  __shared__ CSum shc[DIAG_TPB / 32];
  const CSum a = block_csum<DIAG_TPB>(CSum{s1.s, s1.c}, shc);
  const CSum b = block_csum<DIAG_TPB>(CSum{s2.s, s2.c}, shc);
  if (threadIdx.x == 0) {
    part[4 * blockIdx.x] = a.s;
    part[4 * blockIdx.x + 1] = a.c;
    part[4 * blockIdx.x + 2] = b.s;
    part[4 * blockIdx.x + 3] = b.c;
  }
}

__global__ void k_norms_final(const double *part, int nb, double *out) {
  CSum a{0.0, 0.0}, b{0.0, 0.0};
  for (int q = threadIdx.x; q < nb; q += DIAG_TPB) {
    a = csum_add(a, CSum{part[4 * q], part[4 * q + 1]});
    b = csum_add(b, CSum{part[4 * q + 2], part[4 * q + 3]});
  }
  __shared__ CSum shc[DIAG_TPB / 32];
  a = block_csum<DIAG_TPB>(a, shc);
  b = block_csum<DIAG_TPB>(b, shc);
  if (threadIdx.x == 0) {
    out[0] = a.s + a.c;
    out[1] = b.s + b.c;
  }
}

// ------------------------------------------------------------------ refinement (Sec 2.2)
__device__ __forceinline__ void decode(const DomDev &D, long long off, int &i, int &j, int &k) {
  i = (int)(off % D.px) - GX;
  j = (int)((off / D.px) % D.py) - GH;
  k = (int)(off / D.plane) - GH;
}

// Coarse -> fine: fine ghost cells take the covering coarse cell (injection);
// fine ghost corners take the coarse momentum interpolated linearly along each
// axis (coincident points copy).  All four time-level buffers of the fine
// level receive the current coarse values.
template <typename T>
__global__ void k_prolong(const LevelLink *__restrict__ links, int rC) {
  const LevelLink &L = links[blockIdx.y];
  const DomDev &C = *L.dc, &F = *L.df;
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < L.npcell) {
    long long off = L.pcell[t];
    int i, j, k;
    decode(F, off, i, j, k);
    long long pc = pidx(C, (i + L.ox) >> 1, (j + L.oy) >> 1, k >> 1);
    T r = ((const T *)C.f[rC][0])[pc], q = ((const T *)C.f[rC][1])[pc];
    for (int b = 0; b < NBUF; b++) {
      ((T *)F.f[b][0])[off] = r;
      ((T *)F.f[b][1])[off] = q;
    }
  } else if (t < L.npcell + L.npcorn) {
    long long off = L.pcorn[t - L.npcell];
    int I, J, K;
    decode(F, off, I, J, K);
    int X = I + L.ox, Y = J + L.oy;
    int xs[2] = {X >> 1, (X + 1) >> 1}, ys[2] = {Y >> 1, (Y + 1) >> 1}, zs[2] = {K >> 1, (K + 1) >> 1};
    T s0 = 0, s1 = 0, s2 = 0;
    for (int a = 0; a < 2; a++)
      for (int b = 0; b < 2; b++)
        for (int c = 0; c < 2; c++) {
          long long pc = pidx(C, xs[a], ys[b], zs[c]);
          s0 += ((const T *)C.f[rC][2])[pc];
          s1 += ((const T *)C.f[rC][3])[pc];
          s2 += ((const T *)C.f[rC][4])[pc];
        }
    s0 *= T(0.125);
    s1 *= T(0.125);
    s2 *= T(0.125);
    for (int b = 0; b < NBUF; b++) {
      ((T *)F.f[b][2])[off] = s0;
      ((T *)F.f[b][3])[off] = s1;
      ((T *)F.f[b][4])[off] = s2;
    }
  }
}

// Sibling blocks of one level: one thread per listed ghost-shell point copies
// the sibling's value at the two time levels the next step reads (Sec 2.2,
// the same-level copy of the cube-based mesh).  Sources are interior points
// of the siblings and destinations ghost points, so no thread reads what
// another writes.
template <typename T>
__global__ void k_exchange(const DomDev *__restrict__ doms, const XchItem *__restrict__ x, long long n, int r0,
                           int r1) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const XchItem it = x[t];
  const DomDev &D = doms[it.ddom], &S = doms[it.sdom];
  if (it.kind == XCH_COLUMN) {
    const T *su = (const T *)S.ub[r1];
    T *du = (T *)D.ub[r1];
#pragma unroll
    for (int c = 0; c < 3; c++) du[3 * it.dst + c] = su[3 * it.src + c];
    return;
  }
  const int f0 = it.kind == XCH_CELL ? 0 : 2, f1 = it.kind == XCH_CELL ? 2 : NFIELD;
  for (int f = f0; f < f1; f++) {
    ((T *)D.f[r0][f])[it.dst] = ((const T *)S.f[r0][f])[it.src];
    ((T *)D.f[r1][f])[it.dst] = ((const T *)S.f[r1][f])[it.src];
  }
}

// Fine -> coarse: coarse cells near the covered box boundary take the mean of
// the 8 fine cells they contain; coarse corners inside it or on its lateral
// and top faces take the coincident fine corner.  All four time-level
// buffers of the coarse level.
template <typename T>
__global__ void k_restrict(const LevelLink *__restrict__ links, int rF) {
  const LevelLink &L = links[blockIdx.y];
  const DomDev &C = *L.dc, &F = *L.df;
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < L.nrcell) {
    long long off = L.rcell[t];
    int ic, jc, kc;
    decode(C, off, ic, jc, kc);
    T sr = 0, sp = 0;
    for (int dk = 0; dk < 2; dk++)
      for (int dj = 0; dj < 2; dj++)
        for (int di = 0; di < 2; di++) {
          long long pf = pidx(F, 2 * ic - L.ox + di, 2 * jc - L.oy + dj, 2 * kc + dk);
          sr += ((const T *)F.f[rF][0])[pf];
          sp += ((const T *)F.f[rF][1])[pf];
        }
    sr *= T(0.125);
    sp *= T(0.125);
    for (int b = 0; b < NBUF; b++) {
      ((T *)C.f[b][0])[off] = sr;
      ((T *)C.f[b][1])[off] = sp;
    }
  } else if (t < L.nrcell + L.nrcorn) {
    long long off = L.rcorn[t - L.nrcell];
    int Ic, Jc, Kc;
    decode(C, off, Ic, Jc, Kc);
    long long pf = pidx(F, 2 * Ic - L.ox, 2 * Jc - L.oy, 2 * Kc);
    T a = ((const T *)F.f[rF][2])[pf], b_ = ((const T *)F.f[rF][3])[pf], c = ((const T *)F.f[rF][4])[pf];
    for (int b = 0; b < NBUF; b++) {
      ((T *)C.f[b][2])[off] = a;
      ((T *)C.f[b][3])[off] = b_;
      ((T *)C.f[b][4])[off] = c;
    }
  }
}

// Mass and heat flux through one face of the level's current state, with the
// operations of the full-cell stencil (so the two agree bit for bit): the x-face
// of cell (I,j,k) lies between cells I-1 and I, and so on.
template <typename T>
__device__ __forceinline__ void face_fluxes(const DomDev &D, int rC, int ax, int I, int J, int K, T &fm, T &fh) {
  const T *rp = (const T *)D.f[rC][0];
  const T *pp = (const T *)D.f[rC][1];
  const T *M[3] = {(const T *)D.f[rC][2], (const T *)D.f[rC][3], (const T *)D.f[rC][4]};
  const T *rhob = (const T *)D.rhob, *pb = (const T *)D.pb, *thb = (const T *)D.thb, *ipb = (const T *)D.ipb;
  int li = I, lj = J, lk = K;
  int cI[4], cJ[4], cK[4];
  T S;
  if (ax == 0) {
    li = I - 1;
    S = (T)(D.dy * D.dz);
    cI[0] = I; cJ[0] = J; cK[0] = K;
    cI[1] = I; cJ[1] = J + 1; cK[1] = K;
    cI[2] = I; cJ[2] = J; cK[2] = K + 1;
    cI[3] = I; cJ[3] = J + 1; cK[3] = K + 1;
  } else if (ax == 1) {
    lj = J - 1;
    S = (T)(D.dx * D.dz);
    cI[0] = I; cJ[0] = J; cK[0] = K;
    cI[1] = I + 1; cJ[1] = J; cK[1] = K;
    cI[2] = I; cJ[2] = J; cK[2] = K + 1;
    cI[3] = I + 1; cJ[3] = J; cK[3] = K + 1;
  } else {
    lk = K - 1;
    S = (T)(D.dx * D.dy);
    cI[0] = I; cJ[0] = J; cK[0] = K;
    cI[1] = I + 1; cJ[1] = J; cK[1] = K;
    cI[2] = I; cJ[2] = J + 1; cK[2] = K;
    cI[3] = I + 1; cJ[3] = J + 1; cK[3] = K;
  }
  const T *ub = (const T *)D.ub[rC];
  T u[4];
  for (int s = 0; s < 4; s++) {
    T uc[3];
    corner_u(D, rp, M, rhob, ub, cI[s], cJ[s], cK[s], uc);
    u[s] = uc[ax];
  }
  T ra = cell_rho(D, rp, rhob, li, lj, lk), rb = cell_rho(D, rp, rhob, I, J, K);
  T ta = theta_tot(D, thb, pb, ipb, lk + GH, pp[widx(D, li, lj, lk)]);
  T tb = theta_tot(D, thb, pb, ipb, K + GH, pp[widx(D, I, J, K)]);
  fm = face_flux(ra, rb, u[0], u[1], u[2], u[3], S);
  fh = face_flux(ta, tb, u[0], u[1], u[2], u[3], S);
}

// Flux register: add the fine fluxes of the 2x2 fine faces of every coarse
// interface face, from the fine level's current state (the state its next
// step uses).
template <typename T>
__global__ void k_reg_add(const LevelLink *__restrict__ links, int rF) {
  const LevelLink &L = links[blockIdx.y];
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= L.nfaces) return;
  const IfaceFace f = L.faces[q];
  const DomDev &F = *L.df;
  const int ax = f.ax;
  const T *rp = (const T *)F.f[rF][0];
  const T *pp = (const T *)F.f[rF][1];
  const T *M[3] = {(const T *)F.f[rF][2], (const T *)F.f[rF][3], (const T *)F.f[rF][4]};
  const T *rhob = (const T *)F.rhob, *pb = (const T *)F.pb, *thb = (const T *)F.thb, *ipb = (const T *)F.ipb;
  const T *ub = (const T *)F.ub[rF];
  // the two in-face directions (a, b) of the 2x2 fine faces, as in the face
  // flux of the full-cell stencil: x-face (y, z), y-face (x, z), z-face (x, y)
  const int da_i = ax == 0 ? 0 : 1, da_j = ax == 0 ? 1 : 0, da_k = 0;
  const int db_i = 0, db_j = ax == 2 ? 1 : 0, db_k = ax == 2 ? 0 : 1;
  // normal velocity at the 3x3 corners of the fine faces (one evaluation each)
  T un[3][3];
#pragma unroll
  for (int a = 0; a < 3; a++)
#pragma unroll
    for (int b = 0; b < 3; b++) {
      T uc[3];
      corner_u(F, rp, M, rhob, ub, f.fi + a * da_i + b * db_i, f.fj + a * da_j + b * db_j,
               f.fk + a * da_k + b * db_k, uc);
      un[a][b] = uc[ax];
    }
  const T S = (T)(ax == 0 ? F.dy * F.dz : (ax == 1 ? F.dx * F.dz : F.dx * F.dy));
  const int li = ax == 0 ? -1 : 0, lj = ax == 1 ? -1 : 0, lk = ax == 2 ? -1 : 0;
  T sm = 0, sh = 0;
#pragma unroll
  for (int a = 0; a < 2; a++)
#pragma unroll
    for (int b = 0; b < 2; b++) {
      const int I = f.fi + a * da_i + b * db_i, J = f.fj + a * da_j + b * db_j, K = f.fk + a * da_k + b * db_k;
      T ra = cell_rho(F, rp, rhob, I + li, J + lj, K + lk), rb = cell_rho(F, rp, rhob, I, J, K);
      T ta = theta_tot(F, thb, pb, ipb, K + lk + GH, pp[widx(F, I + li, J + lj, K + lk)]);
      T tb = theta_tot(F, thb, pb, ipb, K + GH, pp[widx(F, I, J, K)]);
      // corners of the face in the full-cell stencil's order: (0,0), (+a), (+b), (+a+b)
      T fm = face_flux(ra, rb, un[a][b], un[a + 1][b], un[a][b + 1], un[a + 1][b + 1], S);
      T fh = face_flux(ta, tb, un[a][b], un[a + 1][b], un[a][b + 1], un[a + 1][b + 1], S);
      sm = Ar<T>::add(sm, fm);
      sh = Ar<T>::add(sh, fh);
    }
  T *rm = (T *)L.regm, *rh = (T *)L.regh;
  rm[q] = Ar<T>::add(rm[q], sm);
  rh[q] = Ar<T>::add(rh[q], sh);
}

template <typename T>
__global__ void k_reg_clear(const LevelLink *__restrict__ links) {
  const LevelLink &L = links[blockIdx.y];
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= L.nfaces) return;
  ((T *)L.regm)[q] = 0;
  ((T *)L.regh)[q] = 0;
}

// Coarse cells next to a refined box: the scalar update of the full-cell
// stencil with the interface faces' fluxes taken from the register (the mean
// over the two fine substeps; cube-boundary flux of Sec 2.2).
template <typename T>
__global__ void k_iface(const LevelLink *__restrict__ links, int rO, int rC, int rN, int rF, int first) {
  const LevelLink &L = links[blockIdx.y];
  using A = Ar<T>;
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= L.nicells) return;
  const IfaceCell ic = L.icells[t];
  const DomDev &D = *L.dc;
  const T dt2 = (T)(first ? D.dt : 2.0 * D.dt);
  const T nu = (T)(first ? 0.0 : D.ra_nu);
  const int i = ic.i, j = ic.j, k = ic.k;
  const T *rm_ = (const T *)L.regm, *rh_ = (const T *)L.regh;
  const T *rp = (const T *)D.f[rC][0];
  const T *pp = (const T *)D.f[rC][1];
  const T *M[3] = {(const T *)D.f[rC][2], (const T *)D.f[rC][3], (const T *)D.f[rC][4]};
  const T *rhob_ = (const T *)D.rhob, *pbv = (const T *)D.pb, *thbv = (const T *)D.thb, *ipbv = (const T *)D.ipb;
  const T *ub = (const T *)D.ub[rC];
  // the eight corner velocities of the cell, [dk][dj][di], and the totals of
  // the cell and its six neighbours (the operations of the full-cell stencil)
  T uc8[2][2][2][3];
#pragma unroll
  for (int dk = 0; dk < 2; dk++)
#pragma unroll
    for (int dj = 0; dj < 2; dj++)
#pragma unroll
      for (int di = 0; di < 2; di++) corner_u(D, rp, M, rhob_, ub, i + di, j + dj, k + dk, uc8[dk][dj][di]);
  const T r0 = cell_rho(D, rp, rhob_, i, j, k);
  const T t0 = theta_tot(D, thbv, pbv, ipbv, k + GH, pp[widx(D, i, j, k)]);
  const T Sf[3] = {(T)(D.dy * D.dz), (T)(D.dx * D.dz), (T)(D.dx * D.dy)};
  T fl[6], hl[6];
#pragma unroll
  for (int ax = 0; ax < 3; ax++)
#pragma unroll
    for (int sd = 0; sd < 2; sd++) {
      int sl = ic.slot[ax * 2 + sd];
      T fm, fh;
      if (sl >= 0) {
        fm = A::mul(T(0.5), rm_[sl]);
        fh = A::mul(T(0.5), rh_[sl]);
      } else {
        const int ni = i + (ax == 0 ? 2 * sd - 1 : 0), nj = j + (ax == 1 ? 2 * sd - 1 : 0),
                  nk = k + (ax == 2 ? 2 * sd - 1 : 0);
        const T rn = cell_rho(D, rp, rhob_, ni, nj, nk);
        const T tn = theta_tot(D, thbv, pbv, ipbv, nk + GH, pp[widx(D, ni, nj, nk)]);
        const T *u0, *u1, *u2, *u3;  // the face's corners in the full-cell stencil's order
        if (ax == 0) {
          u0 = uc8[0][0][sd]; u1 = uc8[0][1][sd]; u2 = uc8[1][0][sd]; u3 = uc8[1][1][sd];
        } else if (ax == 1) {
          u0 = uc8[0][sd][0]; u1 = uc8[0][sd][1]; u2 = uc8[1][sd][0]; u3 = uc8[1][sd][1];
        } else {
          u0 = uc8[sd][0][0]; u1 = uc8[sd][0][1]; u2 = uc8[sd][1][0]; u3 = uc8[sd][1][1];
        }
        // lower-index cell first
        const T ra = sd ? r0 : rn, rb = sd ? rn : r0, ta = sd ? t0 : tn, tb = sd ? tn : t0;
        fm = face_flux(ra, rb, u0[ax], u1[ax], u2[ax], u3[ax], Sf[ax]);
        fh = face_flux(ta, tb, u0[ax], u1[ax], u2[ax], u3[ax], Sf[ax]);
      }
      fl[ax * 2 + sd] = fm;
      hl[ax * 2 + sd] = fh;
    }
  if (k == 0) { fl[4] = 0; hl[4] = 0; }
  if (D.lid && k == D.nz - 1) { fl[5] = 0; hl[5] = 0; }
  T RM = A::add(A::add(A::sub(fl[1], fl[0]), A::sub(fl[3], fl[2])), A::sub(fl[5], fl[4]));
  T RH = A::add(A::add(A::sub(hl[1], hl[0]), A::sub(hl[3], hl[2])), A::sub(hl[5], hl[4]));
  const T *ppO = (const T *)D.f[rO][1];
  const T *rhobp = (const T *)D.pb, *thb = (const T *)D.thb, *pik = (const T *)D.pik, *ipb = (const T *)D.ipb;
  auto tho = [&](int ii, int jj, int kk) { return theta_pert(D, thb, rhobp, ipb, kk + GH, ppO[widx(D, ii, jj, kk)]); };
  T dd = scalar_diffusion<T>(D.dcol[qidx(D, i, j)], k, tho, i, j);
  T Dth = -(T)D.kdif * dd;
  const T v0inv = (T)(1.0 / (D.dx * D.dy * D.dz));
  long long o = pidx(D, i, j, k);
  T rC_ = ((const T *)D.f[rC][0])[o], pC_ = ((const T *)D.f[rC][1])[o];
  T rO_ = ((const T *)D.f[rO][0])[o], pO_ = ppO[o];
  T rN_ = rO_ - dt2 * (RM * v0inv);
  T pN_ = pO_ - dt2 * (T)D.Cp * exner_fac(D, pik, rhobp, ipb, k + GH, pC_) * (RH * v0inv - Dth);
  if (k < D.kug[qidx(D, i, j)]) { rN_ = 0; pN_ = 0; }
  T rF_ = rC_ + nu * (rN_ - T(2) * rC_ + rO_);
  T pF_ = pC_ + nu * (pN_ - T(2) * pC_ + pO_);
  if (k < D.kug[qidx(D, i, j)]) { rF_ = 0; pF_ = 0; }
  ((T *)D.f[rN][0])[o] = rN_;
  ((T *)D.f[rN][1])[o] = pN_;
  ((T *)D.f[rF][0])[o] = rF_;
  ((T *)D.f[rF][1])[o] = pF_;
}

// Two-level perturbation mass of the active cells of one level (a box of
// covered cells excluded), Neumaier-compensated, fixed reduction order.
template <typename T>
__global__ void k_mass_active(const DomDev *__restrict__ dom, int rC, int rO, int both, int bx0, int bx1, int by0,
                              int by1, int bz1, double *part) {
  const DomDev &D = *dom;
  const T *r1 = (const T *)D.f[rC][0], *r0 = (const T *)D.f[rO][0];
  const double V0 = D.dx * D.dy * D.dz;
  long long n = (long long)D.nx * D.ny * D.nz;
  NSum<double> acc{0, 0};
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    int i = (int)(t % D.nx), j = (int)((t / D.nx) % D.ny), k = (int)(t / ((long long)D.nx * D.ny));
    if (i >= bx0 && i < bx1 && j >= by0 && j < by1 && k < bz1) continue;
    const long long o = pidx(D, i, j, k);
    // every member of a merge group carries the group's perturbation, so the
    // cell sum of vf V0 rho' is the group sum of V_G rho'
    double m = (double)r1[o] + (both ? (double)r0[o] : 0.0);
    acc.add(D.vf[t] * V0 * m);
  }
  __shared__ CSum shc[DIAG_TPB / 32];
  const CSum ms = block_csum<DIAG_TPB>(CSum{acc.s, acc.c}, shc);
  if (threadIdx.x == 0) {
    part[5 * blockIdx.x + 0] = ms.s;
    part[5 * blockIdx.x + 1] = ms.c;
    part[5 * blockIdx.x + 2] = 0;
    part[5 * blockIdx.x + 3] = 0;
    part[5 * blockIdx.x + 4] = 0;
  }
}

// ------------------------------------------------------------------ launchers
namespace {
template <typename T, int TYv>
size_t full_smem() {
  return sizeof(FullSmem<T, FullCfg<T, TYv>::PL>);
}

template <typename T, int TYv>
cudaError_t full_t(const StepLaunch &L, int rO, int rC, int rN, int rF, int first, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_full<T, TYv>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)full_smem<T, TYv>());
    if (e != cudaSuccess) return e;
    attr = true;
  }
  if (L.nitems > 0)
    k_full<T, TYv><<<L.nitems, TILE_X * TYv, full_smem<T, TYv>(), st>>>(L.d_doms, L.items, rO, rC, rN, rF,
                                                                        first, L.eos, L.watch);
  // (FP64 lists are not split; this kernel reads cyclic neighbours itself)
  if (L.nwitems > 0)
    k_full<T, TYv><<<L.nwitems, TILE_X * TYv, full_smem<T, TYv>(), st>>>(L.d_doms, L.witems, rO, rC, rN, rF,
                                                                         first, L.eos, L.watch);
  return cudaGetLastError();
}

// the shared memory of k_pair; TMA: raw slots of whole 128-byte lines, plus
// 128 bytes to start the rings on a line
template <int TYv, bool TMA>
size_t pair_smem() {
  using C = PairCfg<TYv>;
  return TMA ? sizeof(PairSmem<C::PL, C::PLP>) + 128 : sizeof(PairSmem<C::PL, C::PL>);
}

// the items of refined boxes (TMA), then those of periodic domains (gather),
// with NR warp roles per block
template <int TYv, int NR>
cudaError_t pair_r(const StepLaunch &L, int rO, int rC, int rN, int rF, int first, cudaStream_t st) {
  if (L.nitems > 0)
    k_pair<TYv, true, NR><<<L.nitems, PairCfg<TYv, NR>::NTH, pair_smem<TYv, true>(), st>>>(
        L.d_doms, L.items, L.tmaps, rO, rC, rN, rF, first, L.eos, L.watch, L.stall_tx);
  if (L.nwitems > 0)
    k_pair<TYv, false, NR><<<L.nwitems, PairCfg<TYv, NR>::NTH, pair_smem<TYv, false>(), st>>>(
        L.d_doms, L.witems, L.tmaps, rO, rC, rN, rF, first, L.eos, L.watch, 0u);
  return cudaGetLastError();
}
template <int TYv>
cudaError_t pair_t(const StepLaunch &L, int rO, int rC, int rN, int rF, int first, cudaStream_t st) {
  if (!L.tmaps) return cudaErrorInvalidValue;
  if (L.roles == 2) return pair_r<TYv, 2>(L, rO, rC, rN, rF, first, st);
  if (L.roles != 1) return cudaErrorInvalidValue;
  return pair_r<TYv, 1>(L, rO, rC, rN, rF, first, st);
}

template <typename T>
cudaError_t groups_t(const StepLaunch &L, int rO, int rC, int rN, int rF, int first, cudaStream_t st) {
  if (L.ngroups > 0)
    k_groups<T><<<(L.ngroups + 127) / 128, 128, 0, st>>>(L.d_doms, L.groups, L.ngroups, L.members, rO, rC, rN,
                                                          rF, first);
  return cudaGetLastError();
}
}  // namespace

int sched_tile_y(int prec, int s) { return prec == CC_FP64 ? SCHED_TY_F64[s] : SCHED_TY_F32[s]; }

cudaError_t launch_exchange(const DomDev *d_doms, const XchItem *items, long long n, int prec, int r0, int r1,
                            cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const unsigned blocks = (unsigned)((n + 255) / 256);
  if (prec == CC_FP64)
    k_exchange<double><<<blocks, 256, 0, st>>>(d_doms, items, n, r0, r1);
  else
    k_exchange<float><<<blocks, 256, 0, st>>>(d_doms, items, n, r0, r1);
  return cudaGetLastError();
}

cudaError_t full_prepare(int prec) {
  auto set = [](auto kern, size_t bytes) {
    return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  };
  cudaError_t e;
  if (prec == CC_FP64) {
    if ((e = set(k_full<double, 8>, full_smem<double, 8>())) != cudaSuccess) return e;
    return set(k_full<double, 4>, full_smem<double, 4>());
  }
  if ((e = set(k_pair<16, true, 1>, pair_smem<16, true>())) != cudaSuccess) return e;
  if ((e = set(k_pair<16, false, 1>, pair_smem<16, false>())) != cudaSuccess) return e;
  if ((e = set(k_pair<8, true, 1>, pair_smem<8, true>())) != cudaSuccess) return e;
  if ((e = set(k_pair<8, false, 1>, pair_smem<8, false>())) != cudaSuccess) return e;
  if ((e = set(k_pair<16, true, 2>, pair_smem<16, true>())) != cudaSuccess) return e;
  if ((e = set(k_pair<16, false, 2>, pair_smem<16, false>())) != cudaSuccess) return e;
  if ((e = set(k_pair<8, true, 2>, pair_smem<8, true>())) != cudaSuccess) return e;
  return set(k_pair<8, false, 2>, pair_smem<8, false>());
}

cudaError_t launch_base(const DomDev &D, int prec, double theta0, double N, double p_surf, double sponge_frac,
                        double tau_max, cudaStream_t st) {
  unsigned nb = (unsigned)((D.pz + 127) / 128);
  if (prec == CC_FP64)
    k_base<double><<<nb, 128, 0, st>>>(D, theta0, N, p_surf, sponge_frac, tau_max, (double *)D.rhob,
                                       (double *)D.pb, (double *)D.thb, (double *)D.pik, (double *)D.rhobc,
                                       (double *)D.tau, (double *)D.ipb);
  else
    k_base<float><<<nb, 128, 0, st>>>(D, theta0, N, p_surf, sponge_frac, tau_max, (float *)D.rhob,
                                      (float *)D.pb, (float *)D.thb, (float *)D.pik, (float *)D.rhobc,
                                      (float *)D.tau, (float *)D.ipb);
  return cudaGetLastError();
}

cudaError_t launch_full(const StepLaunch &L, int prec, int rO, int rC, int rN, int rF, int first,
                        cudaStream_t st) {
  if (prec == CC_FP64) {
    if (L.ty == 8) return full_t<double, 8>(L, rO, rC, rN, rF, first, st);
    if (L.ty == 4) return full_t<double, 4>(L, rO, rC, rN, rF, first, st);
  } else {
    // FP32: two cells per thread with packed arithmetic
    if (L.ty == 16) return pair_t<16>(L, rO, rC, rN, rF, first, st);
    if (L.ty == 8) return pair_t<8>(L, rO, rC, rN, rF, first, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_groups(const StepLaunch &L, int prec, int rO, int rC, int rN, int rF, int first,
                          cudaStream_t st) {
  return prec == CC_FP64 ? groups_t<double>(L, rO, rC, rN, rF, first, st)
                         : groups_t<float>(L, rO, rC, rN, rF, first, st);
}

cudaError_t launch_diagnose(const StepLaunch &L, int prec, int rV, int rC, int rO, int rF, int first, int filter,
                            cudaStream_t st) {
  if (L.ncols <= 0) return cudaSuccess;
  if (prec == CC_FP64)
    k_diag<double><<<(L.ncols + 127) / 128, 128, 0, st>>>(L.d_doms, L.cols, L.ncols, rV, rC, rO, rF, first, filter);
  else
    k_diag<float><<<(L.ncols + 127) / 128, 128, 0, st>>>(L.d_doms, L.cols, L.ncols, rV, rC, rO, rF, first, filter);
  return cudaGetLastError();
}

cudaError_t launch_init_momentum(const DomDev &D, const DomDev *d_dom, int prec, int r, double U, cudaStream_t st) {
  long long n = (long long)(D.ci1 - D.qi0) * (D.cj1 - D.qj0) * D.ck1;
  unsigned nb = (unsigned)((n + 255) / 256);
  if (prec == CC_FP64) k_init_momentum<double><<<nb, 256, 0, st>>>(d_dom, r, U);
  else k_init_momentum<float><<<nb, 256, 0, st>>>(d_dom, r, U);
  return cudaGetLastError();
}

cudaError_t launch_diag_reduce(const DomDev &D, const DomDev *d_dom, int prec, int r, double *d_out,
                               cudaStream_t st) {
  double *part = d_out + 8;
  if (prec == CC_FP64) k_diag_partial<double><<<DIAG_BLOCKS, DIAG_TPB, 0, st>>>(d_dom, r, part);
  else k_diag_partial<float><<<DIAG_BLOCKS, DIAG_TPB, 0, st>>>(d_dom, r, part);
  k_diag_final<<<1, DIAG_TPB, 0, st>>>(part, DIAG_BLOCKS, d_out);
  return cudaGetLastError();
}


namespace {
inline unsigned nb256(long long n) { return (unsigned)((n + 255) / 256); }
}

cudaError_t launch_derived(const DomDev &D, const DomDev *d_dom, int prec, int r, int which, double *d_out,
                           cudaStream_t st) {
  long long n = (long long)D.nx * D.ny * (which == 3 ? D.nz : D.nz + 1);
  if (prec == CC_FP64) k_derived<double><<<nb256(n), 256, 0, st>>>(d_dom, r, which, d_out);
  else k_derived<float><<<nb256(n), 256, 0, st>>>(d_dom, r, which, d_out);
  return cudaGetLastError();
}

cudaError_t launch_norms(const DomDev *a, int prec_a, int ra, const DomDev *b, int prec_b, int rb, int which, int p,
                         int q, int kmin, double *d_out, double *d_part, cudaStream_t st) {
  if (prec_a == CC_FP64 && prec_b == CC_FP64)
    k_norms<double, double><<<DIAG_BLOCKS, DIAG_TPB, 0, st>>>(a, ra, b, rb, which, p, q, kmin, d_part);
  else if (prec_a == CC_FP64)
    k_norms<double, float><<<DIAG_BLOCKS, DIAG_TPB, 0, st>>>(a, ra, b, rb, which, p, q, kmin, d_part);
  else if (prec_b == CC_FP64)
    k_norms<float, double><<<DIAG_BLOCKS, DIAG_TPB, 0, st>>>(a, ra, b, rb, which, p, q, kmin, d_part);
  else
    k_norms<float, float><<<DIAG_BLOCKS, DIAG_TPB, 0, st>>>(a, ra, b, rb, which, p, q, kmin, d_part);
  k_norms_final<<<1, DIAG_TPB, 0, st>>>(d_part, DIAG_BLOCKS, d_out);
  return cudaGetLastError();
}

cudaError_t launch_heat(const DomDev *d_dom, int prec, int r, double *d_out, double *d_part, cudaStream_t st) {
  if (prec == CC_FP64) k_heat_partial<double><<<DIAG_BLOCKS, DIAG_TPB, 0, st>>>(d_dom, r, d_part);
  else k_heat_partial<float><<<DIAG_BLOCKS, DIAG_TPB, 0, st>>>(d_dom, r, d_part);
  k_heat_final<<<1, DIAG_TPB, 0, st>>>(d_part, DIAG_BLOCKS, d_out);
  return cudaGetLastError();
}

// One launch per operation for all the links of a level (its blocks): grid
// rows (blockIdx.y) select the link, columns cover the longest list.
namespace {
dim3 link_grid(const LinkSet &S, long long n) { return dim3(nb256(n), (unsigned)S.n); }
}  // namespace

cudaError_t launch_prolong(const LinkSet &S, int prec, int rC, cudaStream_t st) {
  if (S.n <= 0 || S.maxp <= 0) return cudaSuccess;
  if (prec == CC_FP64) k_prolong<double><<<link_grid(S, S.maxp), 256, 0, st>>>(S.links, rC);
  else k_prolong<float><<<link_grid(S, S.maxp), 256, 0, st>>>(S.links, rC);
  return cudaGetLastError();
}

cudaError_t launch_restrict(const LinkSet &S, int prec, int rF, cudaStream_t st) {
  if (S.n <= 0 || S.maxr <= 0) return cudaSuccess;
  if (prec == CC_FP64) k_restrict<double><<<link_grid(S, S.maxr), 256, 0, st>>>(S.links, rF);
  else k_restrict<float><<<link_grid(S, S.maxr), 256, 0, st>>>(S.links, rF);
  return cudaGetLastError();
}

cudaError_t launch_register_add(const LinkSet &S, int prec, int rF, cudaStream_t st) {
  if (S.n <= 0 || S.maxf <= 0) return cudaSuccess;
  if (prec == CC_FP64) k_reg_add<double><<<link_grid(S, S.maxf), 256, 0, st>>>(S.links, rF);
  else k_reg_add<float><<<link_grid(S, S.maxf), 256, 0, st>>>(S.links, rF);
  return cudaGetLastError();
}

cudaError_t launch_register_clear(const LinkSet &S, int prec, cudaStream_t st) {
  if (S.n <= 0 || S.maxf <= 0) return cudaSuccess;
  if (prec == CC_FP64) k_reg_clear<double><<<link_grid(S, S.maxf), 256, 0, st>>>(S.links);
  else k_reg_clear<float><<<link_grid(S, S.maxf), 256, 0, st>>>(S.links);
  return cudaGetLastError();
}

cudaError_t launch_iface(const LinkSet &S, int prec, int rO, int rC, int rN, int rF, int first, cudaStream_t st) {
  if (S.n <= 0 || S.maxi <= 0) return cudaSuccess;
  if (prec == CC_FP64) k_iface<double><<<link_grid(S, S.maxi), 256, 0, st>>>(S.links, rO, rC, rN, rF, first);
  else k_iface<float><<<link_grid(S, S.maxi), 256, 0, st>>>(S.links, rO, rC, rN, rF, first);
  return cudaGetLastError();
}

cudaError_t launch_mass_active(const DomDev &D, const DomDev *d_dom, int prec, int rC, int rO, int both, int bx0,
                               int bx1, int by0, int by1, int bz1, double *d_out, cudaStream_t st) {
  double *part = d_out + 8;
  if (prec == CC_FP64)
    k_mass_active<double><<<DIAG_BLOCKS, DIAG_TPB, 0, st>>>(d_dom, rC, rO, both, bx0, bx1, by0, by1, bz1, part);
  else
    k_mass_active<float><<<DIAG_BLOCKS, DIAG_TPB, 0, st>>>(d_dom, rC, rO, both, bx0, bx1, by0, by1, bz1, part);
  k_diag_final<<<1, DIAG_TPB, 0, st>>>(part, DIAG_BLOCKS, d_out);
  return cudaGetLastError();
}

}  // namespace cc
