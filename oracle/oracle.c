/*
 * Plain FP64 CPU oracle for the cut-cell finite-volume step of Yamazaki,
 * Satomura & Nikiforakis, "3D cut-cell modelling for high-resolution
 * atmospheric simulations" (arXiv 1509.02572).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * reference that the CUDA path is checked against.  Only the tests, the
 * smoke check and the CPU-baseline leg of the benchmark may load it.  It
 * shares no code, header, table or constant with the CUDA library.
 *
 * What it computes, in the paper's order (section numbers of the paper):
 *   Sec 2.2  block-structured levels with H(l) = 2^-l H and dt(l) = 2^-l dt,
 *            finest level first, two fine steps per coarse step, ghost cells
 *            filled by injection (coarse -> fine) and 8-cell means
 *            (fine -> coarse), two ghost layers integrated by the fine level,
 *            the cube-boundary flux register.
 *   Sec 2.3  bilinear terrain per grid column (Eq. bilin and its four
 *            coefficients), cut-cell volumes and face apertures, the column
 *            gradients (Eqs. xgrad, ygrad), the merge criterion and the merge
 *            direction of the Fig. 6 pseudocode, the semi-staggered variable
 *            arrangement (Fig. 7).
 *   Sec 2.4  finite-volume divergence (Eqs. gauss .. fvm_d), the discrete
 *            momentum / pressure / density equations for uncut cells
 *            (Eqs. momentum_u_d .. continuity form), the cut-cell scalar
 *            fluxes (Eqs. ux1 .. ux3 and the first-order face scalar), the
 *            three-step velocity: prediction on regular velocity cells,
 *            free-slip boundary velocity by normal projection (Eq. 33 and the
 *            nearest-plane interpolation), merged-face interpolation
 *            (gamma / zeta weights).
 *   leapfrog with the Robert-Asselin filter (Sec 2.2).
 *
 * A level is a padded box of cells.  A periodic level wraps its lateral
 * indices (cyclic boundaries, Sec 3); a box level (a refined region) reads
 * its ghost frame, which the multi-level driver fills, and integrates two
 * ghost layers itself.  Readings of points the paper leaves open are listed in
 * the design notes and noted where they apply.
 *
 * Volumes and apertures use exact integration of the bilinear surface
 * (closed form along every vertical face, piecewise Gauss-Legendre over
 * smooth x-segments inside a column), exact for planar terrain.
 *
 * Parity pins: tests/test_oracle_*.py.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "oracle.h"

#define G 4      /* padding of every level array, in cells, on each side */
#define HGZ 2    /* corner levels below the floor / above the lid in host arrays */

enum { C_UG = 0, C_FULL = 1, C_CUT = 2, C_ABS = 3 };    /* cell classes   */
enum { V_UG = 0, V_PRED = 1, V_MF = 2, V_LID = 3 };     /* corner classes */

struct oc_model {
  oc_params P;
  int nx, ny, nz;
  int periodic;       /* lateral indices wrap (cyclic boundaries)          */
  int lid;            /* the top is the rigid lid (else a refinement face) */
  int nxp, nyp, nzp;  /* padded extents                                     */
  long np;            /* nxp*nyp*nzp: cells and corners share the index   */
  long nq;            /* nxp*nyp: columns                                  */
  /* computed region: cells (i,j,k) with ci0<=i<ci1, cj0<=j<cj1, 0<=k<ck1;
   * corner columns (I,J) with qi0<=I<ci1, qj0<=J<cj1 (a box level integrates
   * the corners -1 .. n+1, symmetric about its centre) */
  int ci0, ci1, cj0, cj1, ck1, qi0, qj0;
  /* geometry region (cells whose geometry is evaluated) */
  int gi0, gi1, gj0, gj1, gk1;
  /* terrain */
  double *h;          /* periodic: nx*ny; box: (nxp+1)*(nyp+1), corners -G..n+G */
  double *hc, *gx, *gy;
  double *vf, *ax, *ay, *az;
  int8_t *cls;
  long *target, *root;
  double *vg;
  long *gstart, *gmem;
  int8_t *vcls;
  int32_t *bK, *bI, *bJ; double *ba, *bb, *bn;
  int32_t *mK; double *mg;
  /* base state */
  double *rhob, *pb, *thb; int boff, nb;
  double *rhobc, *tau;  /* per padded corner level */
  /* state: 0 = old (filtered n-1), 1 = current n, 2 = new n+1, 3 = filtered n */
  double *rp[4], *pp[4], *mx[4], *my[4], *mz[4];
  double *ub[4];
  /* work */
  double *rho_t, *th_t, *thp_o, *vel, *RM, *RH;
  /* face fluxes of the last step (mass, heat), indexed by the cell on the
   * high side of the face: the x-face of cell (I,j,k) is x = I dx */
  double *fmx, *fmy, *fmz, *fhx, *fhy, *fhz;
  /* flux-register overrides (refinement): flag and values per face */
  int8_t *ovx, *ovy, *ovz;
  double *ovmx, *ovmy, *ovmz, *ovhx, *ovhy, *ovhz;
  int nsteps;
};

/* ------------------------------------------------------------------ */
/* indexing                                                           */
static inline int wrap(int i, int n) { int r = i % n; return r < 0 ? r + n : r; }
static inline long CI(const oc_model *m, int i, int j, int k) {
  if (m->periodic) { i = wrap(i, m->nx); j = wrap(j, m->ny); }
  return ((long)(k + G) * m->nyp + (j + G)) * m->nxp + (i + G);
}
static inline long QI(const oc_model *m, int i, int j) {
  if (m->periodic) { i = wrap(i, m->nx); j = wrap(j, m->ny); }
  return (long)(j + G) * m->nxp + (i + G);
}
static inline double HC(const oc_model *m, int I, int J) {
  if (m->periodic) return m->h[(long)wrap(J, m->ny) * m->nx + wrap(I, m->nx)];
  return m->h[(long)(J + G) * (m->nxp + 1) + (I + G)];
}
/* interior cell id (k*ny + j)*nx + i of an interior padded index */
static inline long cell_id(const oc_model *m, long p) {
  long i = p % m->nxp - G, j = (p / m->nxp) % m->nyp - G, k = p / m->nq - G;
  return (k * m->ny + j) * m->nx + i;
}
static inline int in_comp_col(const oc_model *m, int I, int J) {
  return I >= m->qi0 && I < m->ci1 && J >= m->qj0 && J < m->cj1;
}
/* highest corner level written by the velocity diagnosis */
static inline int diag_top(const oc_model *m) { return m->lid ? m->nz + G - 1 : m->ck1 - 1; }

/* ------------------------------------------------------------------ */
/* Gauss-Legendre 8-point rule on [-1,1] (standard published nodes).  */
static const double GL_X[4] = {0.1834346424956498049394761, 0.5255324099163289858177390,
                               0.7966664774136267395915539, 0.9602898564975362316835609};
static const double GL_W[4] = {0.3626837833783619829651504, 0.3137066458778872873379622,
                               0.2223810344533744705443560, 0.1012285362903762591525314};

double oc_gauss_legendre8(double (*f)(double, void *), void *ctx, double a, double b) {
  double mid = 0.5 * (a + b), half = 0.5 * (b - a), s = 0.0;
  for (int q = 0; q < 4; q++) {
    s += GL_W[q] * (f(mid - half * GL_X[q], ctx) + f(mid + half * GL_X[q], ctx));
  }
  return s * half;
}

/* ------------------------------------------------------------------ */
/* Geometry of one grid column (Sec 2.3).                             */

/* Integral over s in [0,len] of max(z - h(s), 0) where h is linear from ha to hb. */
double oc_line_int(double z, double ha, double hb, double len) {
  double lo = ha < hb ? ha : hb, hi = ha < hb ? hb : ha;
  if (z >= hi) return len * (z - 0.5 * (ha + hb));
  if (z <= lo) return 0.0;
  double d = z - lo;
  return len * d * d / (2.0 * (hi - lo));
}

/* Fraction of [0,len] where the linear h lies strictly below z. */
double oc_line_frac(double z, double ha, double hb) {
  double lo = ha < hb ? ha : hb, hi = ha < hb ? hb : ha;
  if (lo == hi) return z > lo ? 1.0 : 0.0;
  if (z >= hi) return 1.0;
  if (z <= lo) return 0.0;
  return (z - lo) / (hi - lo);
}

typedef struct { double z, h00, h10, h01, h11, dy; int kind; } colctx;

/* Integrand in x (as s = x/dx in [0,1]) of the column integrals.  At fixed x
 * the bilinear surface is linear in y between h(x,0) and h(x,dy). */
static double col_integrand(double s, void *vctx) {
  colctx *c = (colctx *)vctx;
  double ha = c->h00 + (c->h10 - c->h00) * s;
  double hb = c->h01 + (c->h11 - c->h01) * s;
  if (c->kind == 0) return oc_line_int(c->z, ha, hb, c->dy);
  return oc_line_frac(c->z, ha, hb) * c->dy;
}

/* kind 0: W(z) = integral over the column footprint of max(z - h, 0)
 * kind 1: A(z) = area of the footprint where h < z
 * Integrated in x over segments on which the clipping case does not change
 * (breakpoints where h(x,0) = z, h(x,dy) = z or h(x,0) = h(x,dy)). */
double oc_col_int(double z, double h00, double h10, double h01, double h11, double dx,
                  double dy, int kind) {
  double bp[5];
  int nb = 0;
  bp[nb++] = 0.0;
  if (h10 != h00) {
    double t = (z - h00) / (h10 - h00);
    if (t > 0.0 && t < 1.0) bp[nb++] = t;
  }
  if (h11 != h01) {
    double t = (z - h01) / (h11 - h01);
    if (t > 0.0 && t < 1.0) bp[nb++] = t;
  }
  double den = (h10 - h00) - (h11 - h01);
  if (den != 0.0) {
    double t = (h01 - h00) / den;
    if (t > 0.0 && t < 1.0) bp[nb++] = t;
  }
  bp[nb++] = 1.0;
  /* insertion sort */
  for (int a = 1; a < nb; a++) {
    double v = bp[a];
    int b = a - 1;
    while (b >= 0 && bp[b] > v) { bp[b + 1] = bp[b]; b--; }
    bp[b + 1] = v;
  }
  colctx c = {z, h00, h10, h01, h11, dy, kind};
  double s = 0.0;
  for (int a = 0; a + 1 < nb; a++) {
    if (bp[a + 1] > bp[a]) s += oc_gauss_legendre8(col_integrand, &c, bp[a], bp[a + 1]);
  }
  return s * dx;
}

/* ------------------------------------------------------------------ */
/* Base state (hydrostatic, constant N), reading C-2 of the design notes. */
static void base_state(const oc_params *P, double z, double *rho, double *p) {
  double kap = P->R / P->cp;
  double pis = pow(P->p_surf / P->p0, kap);
  double th, pi;
  if (P->N > 0.0) {
    double n2g = P->N * P->N / P->g;
    th = P->theta0 * exp(n2g * z);
    pi = pis + P->g * P->g / (P->cp * P->theta0 * P->N * P->N) * (exp(-n2g * z) - 1.0);
  } else {
    th = P->theta0;
    pi = pis - P->g * z / (P->cp * P->theta0);
  }
  *p = P->p0 * pow(pi, P->cp / P->R);
  *rho = *p / (P->R * th * pi);
}

/* rho*theta as a function of total pressure: theta = p/(rho R) (p0/p)^(R/cp)
 * (equation of state, Sec 2.1)  =>  rho theta = (p0/R) (p/p0)^(cv/cp). */
static inline double rhotheta_of_p(const oc_params *P, double p) {
  double cv = P->cp - P->R;
  return P->p0 / P->R * pow(p / P->p0, cv / P->cp);
}

/* ------------------------------------------------------------------ */
static void *xcalloc(long n, long sz) { return calloc((size_t)(n > 0 ? n : 1), (size_t)sz); }

void oc_destroy(oc_model *m) {
  if (!m) return;
  void *ptrs[] = {m->h, m->hc, m->gx, m->gy, m->vf, m->ax, m->ay, m->az, m->cls, m->target, m->root,
                  m->vg, m->gstart, m->gmem, m->vcls, m->bK, m->bI, m->bJ, m->ba, m->bb, m->bn, m->mK,
                  m->mg, m->rhob, m->pb, m->thb, m->rhobc, m->tau, m->rho_t, m->th_t, m->thp_o, m->vel,
                  m->RM, m->RH, m->fmx, m->fmy, m->fmz, m->fhx, m->fhy, m->fhz, m->ovx, m->ovy, m->ovz,
                  m->ovmx, m->ovmy, m->ovmz, m->ovhx, m->ovhy, m->ovhz};
  for (size_t i = 0; i < sizeof(ptrs) / sizeof(ptrs[0]); i++) free(ptrs[i]);
  for (int l = 0; l < 4; l++) {
    free(m->rp[l]); free(m->pp[l]); free(m->mx[l]); free(m->my[l]); free(m->mz[l]); free(m->ub[l]);
  }
  free(m);
}

static int build_geometry(oc_model *m);

/* A level: periodic (h has nx*ny corners) or box (h has the padded corner
 * set, (ny+2G+1) rows of (nx+2G+1) corners for I, J = -G .. n+G). */
static oc_model *level_create(const oc_params *P, int periodic, int lid, const double *h, int *status) {
  *status = OC_EINVAL;
  if (P->nx < 4 || P->ny < 4 || P->nz < 4) return NULL;
  oc_model *m = (oc_model *)calloc(1, sizeof(oc_model));
  m->P = *P;
  m->nx = P->nx; m->ny = P->ny; m->nz = P->nz;
  m->periodic = periodic;
  m->lid = lid;
  m->nxp = m->nx + 2 * G; m->nyp = m->ny + 2 * G; m->nzp = m->nz + 2 * G;
  m->nq = (long)m->nxp * m->nyp;
  m->np = m->nq * m->nzp;
  if (periodic) {
    m->ci0 = 0; m->ci1 = m->nx; m->cj0 = 0; m->cj1 = m->ny;
    m->gi0 = 0; m->gi1 = m->nx; m->gj0 = 0; m->gj1 = m->ny;
  } else {
    m->ci0 = -2; m->ci1 = m->nx + 2; m->cj0 = -2; m->cj1 = m->ny + 2;
    m->gi0 = -G; m->gi1 = m->nx + G; m->gj0 = -G; m->gj1 = m->ny + G;
  }
  m->qi0 = periodic ? 0 : -1;
  m->qj0 = periodic ? 0 : -1;
  m->ck1 = lid ? m->nz : m->nz + 2;
  m->gk1 = lid ? m->nz : m->nz + G;
  long nh = periodic ? (long)m->nx * m->ny : (long)(m->nxp + 1) * (m->nyp + 1);
  m->h = xcalloc(nh, sizeof(double));
  memcpy(m->h, h, sizeof(double) * nh);
  long np = m->np, nq = m->nq;
  m->hc = xcalloc(nq, 8); m->gx = xcalloc(nq, 8); m->gy = xcalloc(nq, 8);
  m->vf = xcalloc(np, 8); m->ax = xcalloc(np, 8); m->ay = xcalloc(np, 8); m->az = xcalloc(np, 8);
  m->cls = xcalloc(np, 1); m->target = xcalloc(np, sizeof(long)); m->root = xcalloc(np, sizeof(long));
  m->vg = xcalloc(np, 8);
  m->gstart = xcalloc(np + 1, sizeof(long)); m->gmem = xcalloc(np, sizeof(long));
  m->vcls = xcalloc(np, 1);
  m->bK = xcalloc(nq, 4); m->bI = xcalloc(nq, 4); m->bJ = xcalloc(nq, 4);
  m->ba = xcalloc(nq, 8); m->bb = xcalloc(nq, 8); m->bn = xcalloc(3 * nq, 8);
  m->mK = xcalloc(np, 4); m->mg = xcalloc(np, 8);
  /* base state at cell levels k in [-G-1, nz+G] */
  m->boff = G + 1;
  m->nb = m->nz + 2 * G + 2;
  m->rhob = xcalloc(m->nb, 8); m->pb = xcalloc(m->nb, 8); m->thb = xcalloc(m->nb, 8);
  for (int kk = 0; kk < m->nb; kk++) {
    int k = kk - m->boff;
    base_state(P, (k + 0.5) * P->dz, &m->rhob[kk], &m->pb[kk]);
    m->thb[kk] = rhotheta_of_p(P, m->pb[kk]);
  }
  m->rhobc = xcalloc(m->nzp, 8); m->tau = xcalloc(m->nzp, 8);
  double ztop = P->ztop > 0.0 ? P->ztop : m->nz * P->dz, zs = ztop * (1.0 - P->sponge_frac);
  for (int KK = 0; KK < m->nzp; KK++) {
    int K = KK - G;
    /* reference momentum density at a corner: mean of the two adjacent cell levels */
    m->rhobc[KK] = 0.5 * (m->rhob[K - 1 + m->boff] + m->rhob[K + m->boff]);
    double z = K * P->dz;
    double t = 0.0;
    if (P->sponge_frac > 0.0 && z > zs && z <= ztop) {
      double s = sin(0.5 * M_PI * (z - zs) / (ztop - zs));
      t = P->tau_max * s * s;
    }
    m->tau[KK] = t;
  }
  for (int l = 0; l < 4; l++) {
    m->rp[l] = xcalloc(np, 8); m->pp[l] = xcalloc(np, 8);
    m->mx[l] = xcalloc(np, 8); m->my[l] = xcalloc(np, 8); m->mz[l] = xcalloc(np, 8);
    m->ub[l] = xcalloc(3 * nq, 8);
  }
  m->rho_t = xcalloc(np, 8); m->th_t = xcalloc(np, 8); m->thp_o = xcalloc(np, 8);
  m->vel = xcalloc(3 * np, 8);
  m->RM = xcalloc(np, 8); m->RH = xcalloc(np, 8);
  m->fmx = xcalloc(np, 8); m->fmy = xcalloc(np, 8); m->fmz = xcalloc(np, 8);
  m->fhx = xcalloc(np, 8); m->fhy = xcalloc(np, 8); m->fhz = xcalloc(np, 8);
  m->ovx = xcalloc(np, 1); m->ovy = xcalloc(np, 1); m->ovz = xcalloc(np, 1);
  m->ovmx = xcalloc(np, 8); m->ovmy = xcalloc(np, 8); m->ovmz = xcalloc(np, 8);
  m->ovhx = xcalloc(np, 8); m->ovhy = xcalloc(np, 8); m->ovhz = xcalloc(np, 8);
  int st = build_geometry(m);
  *status = st;
  if (st != OC_OK) { oc_destroy(m); return NULL; }
  return m;
}

oc_model *oc_create(const oc_params *P, const double *h, int *status) {
  return level_create(P, 1, 1, h, status);
}

/* ------------------------------------------------------------------ */
static int build_geometry(oc_model *m) {
  const oc_params *P = &m->P;
  int nz = m->nz;
  double dx = P->dx, dy = P->dy, dz = P->dz;
  int gi0 = m->gi0, gi1 = m->gi1, gj0 = m->gj0, gj1 = m->gj1, gk1 = m->gk1;

  /* column centre height (bilinear value at the centre = mean of corners) and
   * the column gradients of Eqs. xgrad / ygrad */
  for (int j = gj0; j < gj1; j++)
    for (int i = gi0; i < gi1; i++) {
      double h00 = HC(m, i, j), h10 = HC(m, i + 1, j), h01 = HC(m, i, j + 1), h11 = HC(m, i + 1, j + 1);
      long q = QI(m, i, j);
      m->hc[q] = 0.25 * (h00 + h10 + h01 + h11);
      m->gx[q] = ((h10 + h11) - (h00 + h01)) / (2.0 * dx);
      m->gy[q] = ((h01 + h11) - (h00 + h10)) / (2.0 * dy);
    }

  /* volumes and classes; cells outside the geometry region (below the floor
   * or above the lid) stay class 0 with zero volume */
  for (int k = 0; k < gk1; k++)
    for (int j = gj0; j < gj1; j++)
      for (int i = gi0; i < gi1; i++) {
        long c = CI(m, i, j, k);
        double h00 = HC(m, i, j), h10 = HC(m, i + 1, j), h01 = HC(m, i, j + 1), h11 = HC(m, i + 1, j + 1);
        double hmin = fmin(fmin(h00, h10), fmin(h01, h11));
        double hmax = fmax(fmax(h00, h10), fmax(h01, h11));
        double z0 = k * dz, z1 = (k + 1) * dz;
        m->target[c] = -1;
        if (z1 <= hmin) { m->vf[c] = 0.0; m->cls[c] = C_UG; continue; }
        if (z0 >= hmax) { m->vf[c] = 1.0; m->cls[c] = C_FULL; continue; }
        double w1 = oc_col_int(z1, h00, h10, h01, h11, dx, dy, 0);
        double w0 = oc_col_int(z0, h00, h10, h01, h11, dx, dy, 0);
        m->vf[c] = (w1 - w0) / (dx * dy * dz);
        /* merge criterion (Sec 2.3): centre underground or volume below half */
        double zc = (k + 0.5) * dz;
        int small = (m->hc[QI(m, i, j)] > zc) || (m->vf[c] < 0.5);
        m->cls[c] = small ? C_ABS : C_CUT;
      }

  /* lateral apertures: closed form along each vertical face (h linear there) */
  for (int k = 0; k < gk1; k++)
    for (int j = gj0; j < gj1; j++)
      for (int I = gi0; I < gi1; I++) {
        double z0 = k * dz, z1 = (k + 1) * dz;
        double ha = HC(m, I, j), hb = HC(m, I, j + 1);
        double a;
        if (z0 >= fmax(ha, hb)) a = 1.0;
        else if (z1 <= fmin(ha, hb)) a = 0.0;
        else a = (oc_line_int(z1, ha, hb, dy) - oc_line_int(z0, ha, hb, dy)) / (dy * dz);
        m->ax[CI(m, I, j, k)] = a;
        /* y-face y = j*dy of cell (I, j, k): terrain linear from corner (I,j) to (I+1,j) */
        double ya = HC(m, I, j), yb = HC(m, I + 1, j);
        if (z0 >= fmax(ya, yb)) a = 1.0;
        else if (z1 <= fmin(ya, yb)) a = 0.0;
        else a = (oc_line_int(z1, ya, yb, dx) - oc_line_int(z0, ya, yb, dx)) / (dx * dz);
        m->ay[CI(m, I, j, k)] = a;
      }
  /* horizontal apertures az at (i,j,K) = face z = K dz of column (i,j); the
   * floor (K=0) and the rigid lid (K=nz, lid levels) are walls */
  for (int K = 0; K <= gk1 && K < nz + G; K++)
    for (int j = gj0; j < gj1; j++)
      for (int i = gi0; i < gi1; i++) {
        double a = 0.0;
        if (K > 0 && !(m->lid && K >= nz)) {
          double z = K * dz;
          double h00 = HC(m, i, j), h10 = HC(m, i + 1, j), h01 = HC(m, i, j + 1), h11 = HC(m, i + 1, j + 1);
          double hmin = fmin(fmin(h00, h10), fmin(h01, h11));
          double hmax = fmax(fmax(h00, h10), fmax(h01, h11));
          if (z > hmax) a = 1.0;
          else if (z <= hmin) a = 0.0;
          else a = oc_col_int(z, h00, h10, h01, h11, dx, dy, 1) / (dx * dy);
        }
        m->az[CI(m, i, j, K)] = a;
      }

  /* merge direction, Fig. 6 pseudocode */
  for (int k = 0; k < gk1; k++)
    for (int j = gj0; j < gj1; j++)
      for (int i = gi0; i < gi1; i++) {
        long c = CI(m, i, j, k);
        if (m->cls[c] != C_ABS) continue;
        if (!m->periodic && (i < 0 || i >= m->nx || j < 0 || j >= m->ny)) return OC_EGEOM;
        double gx = m->gx[QI(m, i, j)], gy = m->gy[QI(m, i, j)];
        double agx = fabs(gx), agy = fabs(gy);
        long t;
        if (agx <= 1.0 && agy <= 1.0) {
          if (k + 1 >= gk1) return OC_EGEOM;
          t = CI(m, i, j, k + 1);
        } else if (gx > 1.0 && agx >= agy) {
          t = CI(m, i - 1, j, k);
        } else if (gx < -1.0 && agx >= agy) {
          t = CI(m, i + 1, j, k);
        } else if (gy > 1.0 && agx < agy) {
          t = CI(m, i, j - 1, k);
        } else {
          t = CI(m, i, j + 1, k); /* gy < -1 and |gx| < |gy| */
        }
        m->target[c] = t;
      }
  /* merge groups: follow targets to the representative (host) cell; a chain
   * that ends underground or loops is a geometry failure ("v-shaped valley") */
  for (long c = 0; c < m->np; c++) m->root[c] = -1;
  for (int k = 0; k < gk1; k++)
    for (int j = gj0; j < gj1; j++)
      for (int i = gi0; i < gi1; i++) {
        long c = CI(m, i, j, k);
        if (m->cls[c] == C_UG) continue;
        long r = c;
        int n = 0;
        while (m->cls[r] == C_ABS) {
          r = m->target[r];
          if (++n > 64) return OC_EGEOM;
        }
        if (m->cls[r] == C_UG) return OC_EGEOM;
        m->root[c] = r;
      }
  /* members of each group in ascending cell order, and the group volume */
  for (long c = 0; c <= m->np; c++) m->gstart[c] = 0;
  for (long c = 0; c < m->np; c++)
    if (m->root[c] >= 0) m->gstart[m->root[c] + 1]++;
  for (long c = 0; c < m->np; c++) m->gstart[c + 1] += m->gstart[c];
  {
    long *fill = (long *)xcalloc(m->np, sizeof(long));
    for (long c = 0; c < m->np; c++)
      if (m->root[c] >= 0) {
        long r = m->root[c];
        m->gmem[m->gstart[r] + fill[r]++] = c;
      }
    free(fill);
  }
  for (long r = 0; r < m->np; r++) {
    double v = 0.0;
    for (long a = m->gstart[r]; a < m->gstart[r + 1]; a++) v += m->vf[m->gmem[a]] * dx * dy * dz;
    m->vg[r] = v;
  }

  /* velocity-point classes on corners, Sec 2.3 / Fig. 7 and Sec 2.4 */
  for (int K = -G; K < nz + G; K++)
    for (int J = gj0 + (m->periodic ? 0 : 1); J < gj1; J++)
      for (int I = gi0 + (m->periodic ? 0 : 1); I < gi1; I++) {
        long p = CI(m, I, J, K);
        int8_t v;
        if (K * dz <= HC(m, I, J)) v = V_UG;
        else if (m->lid && K >= nz) v = V_LID;
        else if (K < 1 || K >= gk1) v = V_MF;
        else {
          int own = 1;
          for (int dk = -1; dk <= 0; dk++)
            for (int dj = -1; dj <= 0; dj++)
              for (int di = -1; di <= 0; di++) {
                long c = CI(m, I + di, J + dj, K + dk);
                if (m->cls[c] == C_UG || m->root[c] != c) own = 0;
              }
          v = own ? V_PRED : V_MF;
        }
        m->vcls[p] = v;
      }
  /* the lid rule needs a predicted point just below the lid in every column */
  if (m->lid)
    for (int J = m->qj0; J < m->cj1; J++)
      for (int I = m->qi0; I < m->ci1; I++)
        if (m->vcls[CI(m, I, J, nz - 1)] != V_PRED) return OC_EGEOM;

  /* boundary-point stencils: unit normal from the corner gradients of the
   * column-centre heights, then the nearest plane of predicted points crossed
   * by the normal line (Sec 2.4, nearest-plane construction) */
  int ktopsearch = m->lid ? nz - 1 : m->ck1 - 1;
  for (int J = m->qj0; J < m->cj1; J++)
    for (int I = m->qi0; I < m->ci1; I++) {
      long q = QI(m, I, J);
      double hm = m->hc[QI(m, I - 1, J - 1)], h0m = m->hc[QI(m, I, J - 1)];
      double hm0 = m->hc[QI(m, I - 1, J)], h00 = m->hc[QI(m, I, J)];
      double gxc = ((h0m + h00) - (hm + hm0)) / (2.0 * dx);
      double gyc = ((hm0 + h00) - (hm + h0m)) / (2.0 * dy);
      double nrm = sqrt(gxc * gxc + gyc * gyc + 1.0);
      double nxv = -gxc / nrm, nyv = -gyc / nrm, nzv = 1.0 / nrm;
      m->bn[3 * q] = nxv; m->bn[3 * q + 1] = nyv; m->bn[3 * q + 2] = nzv;
      double hh = HC(m, I, J);
      int K0 = 0;
      while (K0 * dz <= hh) K0++;
      int found = 0;
      for (int K = K0; K < K0 + 8 && K <= ktopsearch; K++) {
        double t = (K * dz - hh) / nzv;
        double xN = I * dx + t * nxv, yN = J * dy + t * nyv;
        double fi = floor(xN / dx), fj = floor(yN / dy);
        int i0 = (int)fi, j0 = (int)fj;
        double a = xN / dx - fi, b = yN / dy - fj;
        if (!m->periodic && (i0 < m->gi0 + 1 || i0 + 1 >= m->gi1 || j0 < m->gj0 + 1 || j0 + 1 >= m->gj1))
          return OC_EGEOM;
        /* every point of the plane that carries a nonzero bilinear weight must
         * be a predicted point (on a grid line only that line is needed) */
        int ok = m->vcls[CI(m, i0, j0, K)] == V_PRED &&
                 (a == 0.0 || m->vcls[CI(m, i0 + 1, j0, K)] == V_PRED) &&
                 (b == 0.0 || m->vcls[CI(m, i0, j0 + 1, K)] == V_PRED) &&
                 (a == 0.0 || b == 0.0 || m->vcls[CI(m, i0 + 1, j0 + 1, K)] == V_PRED);
        if (ok) {
          m->bK[q] = K;
          m->bI[q] = m->periodic ? wrap(i0, m->nx) : i0;
          m->bJ[q] = m->periodic ? wrap(j0, m->ny) : j0;
          m->ba[q] = a; m->bb[q] = b;
          found = 1;
          break;
        }
      }
      if (!found) return OC_EGEOM;
    }
  /* merged-face points: interpolate along the vertical line between the
   * boundary point and the nearest predicted point above */
  for (int K = -G; K < nz + G; K++)
    for (int J = m->qj0; J < m->cj1; J++)
      for (int I = m->qi0; I < m->ci1; I++) {
        long p = CI(m, I, J, K);
        m->mK[p] = -1; m->mg[p] = 0.0;
        if (m->vcls[p] != V_MF || K >= m->ck1) continue;
        int ka = -1;
        for (int K2 = K + 1; K2 <= ktopsearch; K2++)
          if (m->vcls[CI(m, I, J, K2)] == V_PRED) { ka = K2; break; }
        if (ka < 0) return OC_EGEOM;
        double hh = HC(m, I, J);
        m->mK[p] = ka;
        m->mg[p] = (K * dz - hh) / (ka * dz - hh);
      }
  return OC_OK;
}

/* ------------------------------------------------------------------ */
/* Totals used by the flux and momentum formulas: base state at the cell's own
 * height plus the stored perturbation.  A cell below the terrain (or outside
 * the floor/lid) has zero perturbation; an absorbed cell carries the
 * perturbation of its merge group. */
static inline double rhob_k(const oc_model *m, int k) { return m->rhob[k + m->boff]; }
static inline double pb_k(const oc_model *m, int k) { return m->pb[k + m->boff]; }
static inline double thb_k(const oc_model *m, int k) { return m->thb[k + m->boff]; }

static double rho_total(const oc_model *m, int L, int i, int j, int k) {
  return rhob_k(m, k) + m->rp[L][CI(m, i, j, k)];
}

/* corner density: mean total density of the 8 cells around the corner */
static double rho_corner(const oc_model *m, int L, int I, int J, int K) {
  double s = 0.0;
  for (int dk = -1; dk <= 0; dk++)
    for (int dj = -1; dj <= 0; dj++)
      for (int di = -1; di <= 0; di++) s += rho_total(m, L, I + di, J + dj, K + dk);
  return s / 8.0;
}

/* Velocity at a corner used by every flux formula, level L (reading C-13):
 * a corner at or below the terrain takes the boundary-point velocity of its
 * vertical line; every other corner holds momentum / corner density.  Ghost
 * corners of a box level hold values given by the coarser level. */
static void corner_velocity(const oc_model *m, int L, int I, int J, int K, double u[3]) {
  if (K * m->P.dz <= HC(m, I, J) && (m->periodic || in_comp_col(m, I, J))) {
    long q = QI(m, I, J);
    u[0] = m->ub[L][3 * q]; u[1] = m->ub[L][3 * q + 1]; u[2] = m->ub[L][3 * q + 2];
    return;
  }
  long p = CI(m, I, J, K);
  double rc = rho_corner(m, L, I, J, K);
  u[0] = m->mx[L][p] / rc; u[1] = m->my[L][p] / rc; u[2] = m->mz[L][p] / rc;
}

/* ------------------------------------------------------------------ */
/* Three-step velocity, steps 2 and 3 (Sec 2.4), for level L:
 *  boundary points: u_N bilinear in the nearest plane, free-slip projection
 *  (or zero for no-slip); merged-face points: linear in z between the
 *  boundary point and the nearest predicted point above; lid points: free-slip
 *  copy of the point below with zero normal component.  Corners at or below
 *  the terrain hold the boundary velocity as momentum (rho_corner * u_B). */
static void diagnose_velocity(oc_model *m, int L) {
  int nz = m->nz;
  for (int J = m->qj0; J < m->cj1; J++)
    for (int I = m->qi0; I < m->ci1; I++) {
      long q = QI(m, I, J);
      double uN[3] = {0, 0, 0};
      int K = m->bK[q], i0 = m->bI[q], j0 = m->bJ[q];
      double a = m->ba[q], b = m->bb[q];
      double w[4] = {(1 - a) * (1 - b), a * (1 - b), (1 - a) * b, a * b};
      int ci[4] = {i0, i0 + 1, i0, i0 + 1}, cj[4] = {j0, j0, j0 + 1, j0 + 1};
      for (int s = 0; s < 4; s++) {
        if (w[s] == 0.0) continue;
        double u[3];
        long p = CI(m, ci[s], cj[s], K);
        double rc = rho_corner(m, L, ci[s], cj[s], K);
        u[0] = m->mx[L][p] / rc; u[1] = m->my[L][p] / rc; u[2] = m->mz[L][p] / rc;
        for (int d = 0; d < 3; d++) uN[d] += w[s] * u[d];
      }
      double *n = &m->bn[3 * q];
      double ubv[3];
      if (m->P.bc_slip) {
        double un = uN[0] * n[0] + uN[1] * n[1] + uN[2] * n[2];
        for (int d = 0; d < 3; d++) ubv[d] = uN[d] - un * n[d];
      } else {
        ubv[0] = ubv[1] = ubv[2] = 0.0;
      }
      for (int d = 0; d < 3; d++) m->ub[L][3 * q + d] = ubv[d];
    }
  int ktop = diag_top(m);
  for (int J = m->qj0; J < m->cj1; J++)
    for (int I = m->qi0; I < m->ci1; I++) {
      long q = QI(m, I, J);
      for (int K = -G + 1; K <= ktop; K++) {
        long p = CI(m, I, J, K);
        int v = m->vcls[p];
        double u[3];
        if (v == V_PRED) continue;
        if (v == V_UG) {
          for (int d = 0; d < 3; d++) u[d] = m->ub[L][3 * q + d];
        } else if (v == V_LID) {
          long pl = CI(m, I, J, nz - 1);
          double rl = rho_corner(m, L, I, J, nz - 1);
          u[0] = m->mx[L][pl] / rl; u[1] = m->my[L][pl] / rl; u[2] = 0.0;
        } else { /* merged face */
          int ka = m->mK[p];
          double g = m->mg[p];
          long pa = CI(m, I, J, ka);
          double ra = rho_corner(m, L, I, J, ka);
          double ua[3] = {m->mx[L][pa] / ra, m->my[L][pa] / ra, m->mz[L][pa] / ra};
          for (int d = 0; d < 3; d++) u[d] = g * ua[d] + (1.0 - g) * m->ub[L][3 * q + d];
        }
        double rc = rho_corner(m, L, I, J, K);
        m->mx[L][p] = rc * u[0]; m->my[L][p] = rc * u[1]; m->mz[L][p] = rc * u[2];
      }
    }
}

/* ------------------------------------------------------------------ */
void oc_init_state(oc_model *m) {
  const oc_params *P = &m->P;
  for (int l = 0; l < 4; l++) {
    memset(m->rp[l], 0, sizeof(double) * m->np);
    memset(m->pp[l], 0, sizeof(double) * m->np);
    memset(m->mx[l], 0, sizeof(double) * m->np);
    memset(m->my[l], 0, sizeof(double) * m->np);
    memset(m->mz[l], 0, sizeof(double) * m->np);
    memset(m->ub[l], 0, sizeof(double) * 3 * m->nq);
  }
  /* uniform flow U on predicted points; zero perturbations */
  for (int K = -G; K < m->nz + G; K++)
    for (int J = m->qj0; J < m->cj1; J++)
      for (int I = m->qi0; I < m->ci1; I++) {
        long p = CI(m, I, J, K);
        if (m->vcls[p] == V_PRED) m->mx[1][p] = rho_corner(m, 1, I, J, K) * P->U;
      }
  diagnose_velocity(m, 1);
  m->nsteps = 0;
}

/* ------------------------------------------------------------------ */
/* Artificial diffusion (Sec 2.1: fourth order in the horizontal and vertical
 * directions; Sec 2.4: a second-order term, with the boundary conditions of the
 * terrain surface, where the neighbouring fluid points a fourth-order term
 * needs are missing).  Reading C-4, per axis of each point:
 *   fluid points of a scalar stencil: cells owning their pressure point (full
 *     or cut, not absorbed and not below the terrain) inside the level (above
 *     the floor, below the rigid lid);
 *   fluid points of a velocity stencil: corners above the terrain and below
 *     the rigid lid;
 *   all four neighbours at distance 1 and 2 fluid: the fourth difference
 *     f(-2) - 4 f(-1) + 6 f(0) - 4 f(1) + f(2), with D = -K4 * (its sum over
 *     the axes);
 *   otherwise the second difference over the neighbours at distance 1 with
 *     K2 = 4 K4 / d^2 (the same damping of the shortest, 2d, wave), entered as
 *     -4 (f(-1) - 2 f(0) + f(1)) in that sum; a scalar neighbour that is not a
 *     fluid point takes the centre value (no diffusive flux through the wall),
 *     a velocity neighbour that is not a fluid point keeps its stored value
 *     (the boundary-point velocity below the terrain, the free-slip value on
 *     the lid). */
static int cell_fluid(const oc_model *m, int i, int j, int k) {
  if (k < 0 || k >= m->gk1) return 0;
  int c = m->cls[CI(m, i, j, k)];
  return c == C_FULL || c == C_CUT;
}
static int corner_fluid(const oc_model *m, int I, int J, int K) {
  if (K <= 0 || (m->lid && K >= m->nz)) return 0;
  return K * m->P.dz > HC(m, I, J);
}
/* the axis term of the diffusion sum for values f[0..4] at offsets -2..2 with
 * fluid flags fl[0..4]; scalar selects the zero-gradient wall condition */
static double diff_axis(const double f[5], const int fl[5], int scalar) {
  if (fl[0] && fl[1] && fl[3] && fl[4]) return f[0] - 4 * f[1] + 6 * f[2] - 4 * f[3] + f[4];
  double lo = (fl[1] || !scalar) ? f[1] : f[2];
  double hi = (fl[3] || !scalar) ? f[3] : f[2];
  return -4.0 * (lo - 2.0 * f[2] + hi);
}

/* ------------------------------------------------------------------ */
static void scalar_residuals(oc_model *m);

/* Cells of the computed region as (i,j,k) triplets */
#define FOR_COMP(m, i, j, k)                     \
  for (int k = 0; k < (m)->ck1; k++)             \
    for (int j = (m)->cj0; j < (m)->cj1; j++)    \
      for (int i = (m)->ci0; i < (m)->ci1; i++)

/* One leapfrog step.  Level 0 = filtered n-1, 1 = n; writes 2 = n+1 and
 * 3 = filtered n, then rotates so that (0,1) = (filtered n, n+1).
 * The first step is forward Euler: old = current, half the leapfrog interval,
 * no filter (reading C-3).  Values outside the computed region (the ghost
 * frame of a box level, the levels below the floor) are carried over
 * unchanged to both new levels. */
void oc_step(oc_model *m, int nsteps) {
  const oc_params *P = &m->P;
  int nz = m->nz;
  double dx = P->dx, dy = P->dy, dz = P->dz, V0 = dx * dy * dz;
  double kap = P->R / P->cp, Cp = P->cp * P->R / (P->cp - P->R);
  /* cells whose totals / corner velocities are tabulated: the computed region
   * plus its stencil halo */
  int ti0 = m->periodic ? 0 : -G, ti1 = m->periodic ? m->nx : m->nx + G;
  int tj0 = m->periodic ? 0 : -G, tj1 = m->periodic ? m->ny : m->ny + G;
  int ktop = diag_top(m);
  for (int s = 0; s < nsteps; s++) {
    int first = (m->nsteps == 0);
    int O = first ? 1 : 0; /* level used as "n-1" */
    double dt2 = first ? P->dt : 2.0 * P->dt;
    double nu = first ? 0.0 : P->ra_nu;
    double kdif = P->c4 / (16.0 * P->dt);

    /* cell totals at n and the rho-theta perturbation at n-1 */
    for (int k = -G; k < nz + G; k++)
      for (int j = tj0; j < tj1; j++)
        for (int i = ti0; i < ti1; i++) {
          long c = CI(m, i, j, k);
          m->rho_t[c] = rhob_k(m, k) + m->rp[1][c];
          m->th_t[c] = rhotheta_of_p(P, pb_k(m, k) + m->pp[1][c]);
          m->thp_o[c] = rhotheta_of_p(P, pb_k(m, k) + m->pp[O][c]) - thb_k(m, k);
        }
    /* corner velocities at n */
    for (int K = -G + 1; K < nz + G; K++)
      for (int J = tj0 + (m->periodic ? 0 : 1); J < tj1; J++)
        for (int I = ti0 + (m->periodic ? 0 : 1); I < ti1; I++) {
          long p = CI(m, I, J, K);
          corner_velocity(m, 1, I, J, K, &m->vel[3 * p]);
        }
    scalar_residuals(m);

    /* carry every value over; the computed region is overwritten below */
    for (long c = 0; c < m->np; c++) {
      m->rp[2][c] = m->rp[3][c] = m->rp[1][c];
      m->pp[2][c] = m->pp[3][c] = m->pp[1][c];
      m->mx[2][c] = m->mx[3][c] = m->mx[1][c];
      m->my[2][c] = m->my[3][c] = m->my[1][c];
      m->mz[2][c] = m->mz[3][c] = m->mz[1][c];
    }

    /* scalar update per merge group (Sec 2.3/2.4): divergence over the
     * merged volume, host update, scatter to the absorbed cells */
    FOR_COMP(m, ir, jr, kr) {
      long r = CI(m, ir, jr, kr);
      if (m->cls[r] == C_UG) {
        m->rp[2][r] = m->pp[2][r] = m->rp[3][r] = m->pp[3][r] = 0.0;
        continue;
      }
      if (m->root[r] != r) continue;
      double rm = 0.0, rh = 0.0;
      for (long a = m->gstart[r]; a < m->gstart[r + 1]; a++) {
        rm += m->RM[m->gmem[a]]; rh += m->RH[m->gmem[a]];
      }
      double VG = m->vg[r];
      /* artificial diffusion of (rho theta)' at n-1 at the host (reading C-4) */
      double d4 = 0.0;
      {
        double f[5];
        int fl[5];
        for (int a = -2; a <= 2; a++) {
          f[a + 2] = m->thp_o[CI(m, ir + a, jr, kr)];
          fl[a + 2] = cell_fluid(m, ir + a, jr, kr);
        }
        d4 += diff_axis(f, fl, 1);
        for (int a = -2; a <= 2; a++) {
          f[a + 2] = m->thp_o[CI(m, ir, jr + a, kr)];
          fl[a + 2] = cell_fluid(m, ir, jr + a, kr);
        }
        d4 += diff_axis(f, fl, 1);
        for (int a = -2; a <= 2; a++) {
          f[a + 2] = m->thp_o[CI(m, ir, jr, kr + a)];
          fl[a + 2] = cell_fluid(m, ir, jr, kr + a);
        }
        d4 += diff_axis(f, fl, 1);
      }
      double Dth = -kdif * d4;
      double pn = pb_k(m, kr) + m->pp[1][r];
      double rn = m->rp[O][r] - dt2 * rm / VG;
      double pnew = m->pp[O][r] - dt2 * Cp * pow(pn / P->p0, kap) * (rh / VG - Dth);
      double rf = m->rp[1][r] + nu * (rn - 2.0 * m->rp[1][r] + m->rp[O][r]);
      double pf = m->pp[1][r] + nu * (pnew - 2.0 * m->pp[1][r] + m->pp[O][r]);
      /* every member carries the group's perturbation (reading: an absorbed
       * cell's totals are its own base state plus the group perturbation) */
      for (long a = m->gstart[r]; a < m->gstart[r + 1]; a++) {
        long c = m->gmem[a];
        m->rp[2][c] = rn; m->pp[2][c] = pnew;
        m->rp[3][c] = rf; m->pp[3][c] = pf;
      }
    }

    /* momentum on predicted velocity cells, Eqs. momentum_u_d .. w_d */
    FOR_COMP(m, I, J, K) {
      long p = CI(m, I, J, K);
      if (m->vcls[p] != V_PRED || !in_comp_col(m, I, J)) continue;
      double rE = 0, rW = 0, rN = 0, rS = 0, rT = 0, rB = 0;
      double pE = 0, pW = 0, pN = 0, pS = 0, pT = 0, pB = 0, r8 = 0;
      for (int a = -1; a <= 0; a++)
        for (int b = -1; b <= 0; b++) {
          rE += m->rho_t[CI(m, I, J + a, K + b)];
          rW += m->rho_t[CI(m, I - 1, J + a, K + b)];
          rN += m->rho_t[CI(m, I + a, J, K + b)];
          rS += m->rho_t[CI(m, I + a, J - 1, K + b)];
          rT += m->rho_t[CI(m, I + a, J + b, K)];
          rB += m->rho_t[CI(m, I + a, J + b, K - 1)];
          pE += m->pp[1][CI(m, I, J + a, K + b)];
          pW += m->pp[1][CI(m, I - 1, J + a, K + b)];
          pN += m->pp[1][CI(m, I + a, J, K + b)];
          pS += m->pp[1][CI(m, I + a, J - 1, K + b)];
          pT += m->pp[1][CI(m, I + a, J + b, K)];
          pB += m->pp[1][CI(m, I + a, J + b, K - 1)];
          r8 += m->rp[1][CI(m, I + a, J + b, K)] + m->rp[1][CI(m, I + a, J + b, K - 1)];
        }
      rE *= 0.25; rW *= 0.25; rN *= 0.25; rS *= 0.25; rT *= 0.25; rB *= 0.25;
      const double *u0 = &m->vel[3 * p];
      const double *uE = &m->vel[3 * CI(m, I + 1, J, K)], *uW = &m->vel[3 * CI(m, I - 1, J, K)];
      const double *uN = &m->vel[3 * CI(m, I, J + 1, K)], *uS = &m->vel[3 * CI(m, I, J - 1, K)];
      const double *uT = &m->vel[3 * CI(m, I, J, K + 1)], *uB = &m->vel[3 * CI(m, I, J, K - 1)];
      double fE = rE * 0.5 * (u0[0] + uE[0]) * dy * dz, fW = rW * 0.5 * (uW[0] + u0[0]) * dy * dz;
      double fN = rN * 0.5 * (u0[1] + uN[1]) * dx * dz, fS = rS * 0.5 * (uS[1] + u0[1]) * dx * dz;
      double fT = rT * 0.5 * (u0[2] + uT[2]) * dx * dy, fB = rB * 0.5 * (uB[2] + u0[2]) * dx * dy;
      double tend[3];
      for (int d = 0; d < 3; d++) {
        double adv = fE * 0.5 * (u0[d] + uE[d]) - fW * 0.5 * (uW[d] + u0[d]) +
                     fN * 0.5 * (u0[d] + uN[d]) - fS * 0.5 * (uS[d] + u0[d]) +
                     fT * 0.5 * (u0[d] + uT[d]) - fB * 0.5 * (uB[d] + u0[d]);
        tend[d] = -adv / V0;
      }
      tend[0] -= 0.25 * (pE - pW) / dx;
      tend[1] -= 0.25 * (pN - pS) / dy;
      tend[2] -= 0.25 * (pT - pB) / dz;
      tend[2] -= P->g * r8 / 8.0;
      /* diffusion and sponge on the momentum departure from the reference
       * state (rho_bar U, 0, 0), level n-1 (readings C-4, C-5) */
      double *MO[3] = {m->mx[O], m->my[O], m->mz[O]};
      int flx[5], fly[5], flz[5];
      for (int a = -2; a <= 2; a++) {
        flx[a + 2] = corner_fluid(m, I + a, J, K);
        fly[a + 2] = corner_fluid(m, I, J + a, K);
        flz[a + 2] = corner_fluid(m, I, J, K + a);
      }
      for (int d = 0; d < 3; d++) {
        /* reference momentum (rho_bar_corner U, 0, 0) at corner level K */
        double ref0 = d == 0 ? m->rhobc[K + G] * P->U : 0.0;
        double f[5], d4 = 0.0;
        for (int a = -2; a <= 2; a++) f[a + 2] = MO[d][CI(m, I + a, J, K)] - ref0;
        d4 += diff_axis(f, flx, 0);
        for (int a = -2; a <= 2; a++) f[a + 2] = MO[d][CI(m, I, J + a, K)] - ref0;
        d4 += diff_axis(f, fly, 0);
        for (int a = -2; a <= 2; a++)
          f[a + 2] = MO[d][CI(m, I, J, K + a)] - (d == 0 ? m->rhobc[K + a + G] * P->U : 0.0);
        d4 += diff_axis(f, flz, 0);
        tend[d] += -kdif * d4 - m->tau[K + G] * (MO[d][p] - ref0);
      }
      double *MN[3] = {m->mx[2], m->my[2], m->mz[2]};
      for (int d = 0; d < 3; d++) MN[d][p] = MO[d][p] + dt2 * tend[d];
    }
    /* steps 2 and 3 of the velocity calculation on the new level; they need
     * the new densities, so they follow the scalar update */
    diagnose_velocity(m, 2);
    /* Robert-Asselin filter on every corner value of the computed columns
     * (prognostic or diagnosed) */
    for (int K = -G + 1; K <= ktop; K++)
      for (int J = m->qj0; J < m->cj1; J++)
        for (int I = m->qi0; I < m->ci1; I++) {
          long p = CI(m, I, J, K);
          m->mx[3][p] = m->mx[1][p] + nu * (m->mx[2][p] - 2.0 * m->mx[1][p] + m->mx[O][p]);
          m->my[3][p] = m->my[1][p] + nu * (m->my[2][p] - 2.0 * m->my[1][p] + m->my[O][p]);
          m->mz[3][p] = m->mz[1][p] + nu * (m->mz[2][p] - 2.0 * m->mz[1][p] + m->mz[O][p]);
        }
    /* rotate: old <- filtered n, current <- n+1 */
    double *t;
#define ROT(A)                      \
  t = A[0]; A[0] = A[3]; A[3] = t;  \
  t = A[1]; A[1] = A[2]; A[2] = t;
    ROT(m->rp); ROT(m->pp); ROT(m->mx); ROT(m->my); ROT(m->mz); ROT(m->ub);
#undef ROT
    m->nsteps++;
  }
}

/* Face fluxes of mass and rho*theta (Sec 2.4): normal velocity = mean of the
 * four corner velocities of the face (Eqs. ux1-ux3), face scalar = mean of the
 * two cells exchanging the flux, area = aperture * full face area, zero flux
 * through the terrain, floor and lid.  Each cell sums its own outward fluxes;
 * faces inside one merge group are skipped (they cancel in the group sum).
 * A face flagged by the flux register takes the register's value. */
static void scalar_residuals(oc_model *m) {
  const oc_params *P = &m->P;
  int nz = m->nz;
  double dx = P->dx, dy = P->dy, dz = P->dz;
  FOR_COMP(m, i, j, k) {
    long c = CI(m, i, j, k);
    m->RM[c] = 0.0; m->RH[c] = 0.0;
    if (m->cls[c] == C_UG) continue;
    double rm = 0.0, rh = 0.0;
    /* six faces: (axis, side) with side 1 = high face */
    for (int ax = 0; ax < 3; ax++)
      for (int sd = 0; sd <= 1; sd++) {
        int ni = i, nj = j, nk = k;
        double A, S;
        int cI[4], cJ[4], cK[4];
        long fc; /* the cell on the high side of the face */
        if (ax == 0) {
          int I = i + sd;
          ni = i + (sd ? 1 : -1);
          fc = CI(m, I, j, k);
          A = m->ax[fc];
          S = dy * dz;
          int cc[4][3] = {{I, j, k}, {I, j + 1, k}, {I, j, k + 1}, {I, j + 1, k + 1}};
          for (int s = 0; s < 4; s++) { cI[s] = cc[s][0]; cJ[s] = cc[s][1]; cK[s] = cc[s][2]; }
        } else if (ax == 1) {
          int J = j + sd;
          nj = j + (sd ? 1 : -1);
          fc = CI(m, i, J, k);
          A = m->ay[fc];
          S = dx * dz;
          int cc[4][3] = {{i, J, k}, {i + 1, J, k}, {i, J, k + 1}, {i + 1, J, k + 1}};
          for (int s = 0; s < 4; s++) { cI[s] = cc[s][0]; cJ[s] = cc[s][1]; cK[s] = cc[s][2]; }
        } else {
          int K = k + sd;
          nk = k + (sd ? 1 : -1);
          fc = CI(m, i, j, K);
          A = m->az[fc];
          S = dx * dy;
          int cc[4][3] = {{i, j, K}, {i + 1, j, K}, {i, j + 1, K}, {i + 1, j + 1, K}};
          for (int s = 0; s < 4; s++) { cI[s] = cc[s][0]; cJ[s] = cc[s][1]; cK[s] = cc[s][2]; }
        }
        if (A == 0.0) continue;
        if (nk < 0 || (m->lid && nk >= nz)) continue;
        long nc = CI(m, ni, nj, nk);
        if (m->cls[nc] != C_UG && m->root[nc] == m->root[c]) continue;
        int8_t *ov = ax == 0 ? m->ovx : (ax == 1 ? m->ovy : m->ovz);
        double fm, fh;
        if (ov[fc]) {
          fm = (ax == 0 ? m->ovmx : (ax == 1 ? m->ovmy : m->ovmz))[fc];
          fh = (ax == 0 ? m->ovhx : (ax == 1 ? m->ovhy : m->ovhz))[fc];
        } else {
          double un = 0.0;
          for (int s = 0; s < 4; s++) un += m->vel[3 * CI(m, cI[s], cJ[s], cK[s]) + ax];
          un *= 0.25;
          fm = 0.5 * (m->rho_t[c] + m->rho_t[nc]) * un * A * S;
          fh = 0.5 * (m->th_t[c] + m->th_t[nc]) * un * A * S;
        }
        (ax == 0 ? m->fmx : (ax == 1 ? m->fmy : m->fmz))[fc] = fm;
        (ax == 0 ? m->fhx : (ax == 1 ? m->fhy : m->fhz))[fc] = fh;
        if (sd) { rm += fm; rh += fh; } else { rm -= fm; rh -= fh; }
      }
    m->RM[c] = rm; m->RH[c] = rh;
  }
}

/* ------------------------------------------------------------------ */
/* accessors (host layouts: interior cells nz*ny*nx, corners K = -2 .. nz+2) */
static double *level_array(oc_model *m, int field, int level) {
  switch (field) {
    case OC_F_RHOP: return m->rp[level];
    case OC_F_PP: return m->pp[level];
    case OC_F_MX: return m->mx[level];
    case OC_F_MY: return m->my[level];
    case OC_F_MZ: return m->mz[level];
    case OC_F_UB: return m->ub[level];
  }
  return NULL;
}

int oc_dims(const oc_model *m, long *ncell, long *ncorner, long *ncol, int *gz) {
  *ncell = (long)m->nx * m->ny * m->nz;
  *ncorner = (long)m->nx * m->ny * (m->nz + 1 + 2 * HGZ);
  *ncol = (long)m->nx * m->ny;
  *gz = HGZ;
  return OC_OK;
}

static void copy_field(oc_model *m, int field, double *a, double *host, int to_host) {
  int nx = m->nx, ny = m->ny, nz = m->nz;
  if (field == OC_F_UB) {
    for (int j = 0; j < ny; j++)
      for (int i = 0; i < nx; i++)
        for (int d = 0; d < 3; d++) {
          long q = 3 * QI(m, i, j) + d, h = ((long)j * nx + i) * 3 + d;
          if (to_host) host[h] = a[q]; else a[q] = host[h];
        }
    return;
  }
  int k0 = 0, k1 = nz;
  if (field >= OC_F_MX) { k0 = -HGZ; k1 = nz + HGZ + 1; }
  long h = 0;
  for (int k = k0; k < k1; k++)
    for (int j = 0; j < ny; j++)
      for (int i = 0; i < nx; i++, h++) {
        long p = CI(m, i, j, k);
        if (to_host) host[h] = a[p]; else a[p] = host[h];
      }
}

int oc_get_state(oc_model *m, int field, int level, double *out) {
  if (level < 0 || level > 1) return OC_EINVAL;
  double *a = level_array(m, field, level);
  if (!a) return OC_EINVAL;
  copy_field(m, field, a, out, 1);
  return OC_OK;
}

/* The whole padded array of a prognostic field (cells or corners, G = 4
 * layers on every side, index ((k + G) * nyp + j + G) * nxp + i + G), ghost
 * frame included: lets tests check the coarse-fine exchange cell by cell. */
int oc_get_state_padded(oc_model *m, int field, int level, double *out) {
  if (level < 0 || level > 1 || field == OC_F_UB) return OC_EINVAL;
  double *a = level_array(m, field, level);
  if (!a) return OC_EINVAL;
  long n = (long)m->nxp * m->nyp * m->nzp;
  for (long q = 0; q < n; q++) out[q] = a[q];
  return OC_OK;
}

void oc_padding(const oc_model *m, int *g, int *nxp, int *nyp, int *nzp) {
  *g = G; *nxp = m->nxp; *nyp = m->nyp; *nzp = m->nzp;
}

int oc_set_state(oc_model *m, int field, int level, const double *in) {
  if (level < 0 || level > 1) return OC_EINVAL;
  double *a = level_array(m, field, level);
  if (!a) return OC_EINVAL;
  copy_field(m, field, a, (double *)in, 0);
  return OC_OK;
}

int oc_get_geometry(const oc_model *m, double *vf, double *ax, double *ay, double *az, int8_t *cls,
                    int32_t *root, double *vg, double *hc, double *gx, double *gy) {
  int nx = m->nx, ny = m->ny, nz = m->nz;
  long h = 0;
  for (int k = 0; k < nz; k++)
    for (int j = 0; j < ny; j++)
      for (int i = 0; i < nx; i++, h++) {
        long p = CI(m, i, j, k);
        vf[h] = m->vf[p]; ax[h] = m->ax[p]; ay[h] = m->ay[p]; cls[h] = m->cls[p];
        root[h] = m->root[p] >= 0 ? (int32_t)cell_id(m, m->root[p]) : -1;
        vg[h] = m->vg[p];
      }
  h = 0;
  for (int K = 0; K <= nz; K++)
    for (int j = 0; j < ny; j++)
      for (int i = 0; i < nx; i++, h++) az[h] = m->az[CI(m, i, j, K)];
  h = 0;
  for (int j = 0; j < ny; j++)
    for (int i = 0; i < nx; i++, h++) {
      long q = QI(m, i, j);
      hc[h] = m->hc[q]; gx[h] = m->gx[q]; gy[h] = m->gy[q];
    }
  return OC_OK;
}

int oc_get_points(const oc_model *m, int8_t *vcls, int32_t *bK, int32_t *bI, int32_t *bJ, double *ba,
                  double *bb, double *bn, int32_t *mK, double *mg) {
  int nx = m->nx, ny = m->ny, nz = m->nz;
  long h = 0;
  for (int K = -HGZ; K <= nz + HGZ; K++)
    for (int j = 0; j < ny; j++)
      for (int i = 0; i < nx; i++, h++) {
        long p = CI(m, i, j, K);
        vcls[h] = m->vcls[p]; mK[h] = m->mK[p]; mg[h] = m->mg[p];
      }
  h = 0;
  for (int j = 0; j < ny; j++)
    for (int i = 0; i < nx; i++, h++) {
      long q = QI(m, i, j);
      bK[h] = m->bK[q]; bI[h] = m->bI[q]; bJ[h] = m->bJ[q];
      ba[h] = m->ba[q]; bb[h] = m->bb[q];
      for (int d = 0; d < 3; d++) bn[3 * h + d] = m->bn[3 * q + d];
    }
  return OC_OK;
}

int oc_base_len(const oc_model *m) { return m->nb; }

int oc_get_base(const oc_model *m, double *rhob, double *pb, int *koff, int *nb) {
  memcpy(rhob, m->rhob, 8 * m->nb); memcpy(pb, m->pb, 8 * m->nb);
  *koff = m->boff; *nb = m->nb;
  return OC_OK;
}

/* Perturbation mass of the interior: sum over merge groups of V_G * rho'_G. */
double oc_mass(const oc_model *m, int level) {
  double s = 0.0;
  for (int k = 0; k < m->nz; k++)
    for (int j = 0; j < m->ny; j++)
      for (int i = 0; i < m->nx; i++) {
        long c = CI(m, i, j, k);
        if (m->cls[c] != C_UG && m->root[c] == c) s += m->vg[c] * m->rp[level][c];
      }
  return s;
}

int oc_nsteps(const oc_model *m) { return m->nsteps; }

/* Heat content of the interior: sum over merge groups of V_G (rho theta)'_G,
 * where (rho theta)' is rho theta of the total pressure minus that of the
 * base pressure, both from the equation of state (Sec 2.1).  The scheme does
 * not conserve it (the pressure equation is not in flux form); it is a
 * diagnostic. */
double oc_heat(const oc_model *m, int level) {
  double s = 0.0;
  for (int k = 0; k < m->nz; k++)
    for (int j = 0; j < m->ny; j++)
      for (int i = 0; i < m->nx; i++) {
        long c = CI(m, i, j, k);
        if (m->cls[c] != C_UG && m->root[c] == c) {
          double p = pb_k(m, k);
          s += m->vg[c] * (rhotheta_of_p(&m->P, p + m->pp[level][c]) - rhotheta_of_p(&m->P, p));
        }
      }
  return s;
}

/* Derived output fields of time level `level` (0 filtered previous, 1
 * current).  OC_D_U, OC_D_V, OC_D_W (level 1 only: the boundary-point
 * velocity is diagnosed for the current level alone): the corner velocity
 * every flux formula uses (corner_velocity above), corners K = 0 .. nz,
 * (nz+1)*ny*nx values.
 * OC_D_THETA: potential-temperature perturbation of every cell,
 * theta' = (rho theta)(p_bar + p') / (rho_bar + rho') - (rho theta)(p_bar) / rho_bar,
 * nz*ny*nx values (absorbed cells carry their group's state, cells below the
 * terrain give 0). */
int oc_get_derived(const oc_model *m, int which, int level, double *out) {
  if (level < 0 || level > 1 || which < OC_D_U || which > OC_D_THETA) return OC_EINVAL;
  if (which != OC_D_THETA && level != 1) return OC_EINVAL;
  int nx = m->nx, ny = m->ny, nz = m->nz;
  long h = 0;
  if (which == OC_D_THETA) {
    for (int k = 0; k < nz; k++)
      for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++, h++) {
          long c = CI(m, i, j, k);
          double p = pb_k(m, k), r = rhob_k(m, k);
          out[h] = rhotheta_of_p(&m->P, p + m->pp[level][c]) / (r + m->rp[level][c]) -
                   rhotheta_of_p(&m->P, p) / r;
        }
    return OC_OK;
  }
  for (int K = 0; K <= nz; K++)
    for (int J = 0; J < ny; J++)
      for (int I = 0; I < nx; I++, h++) {
        double u[3];
        corner_velocity(m, level, I, J, K, u);
        out[h] = u[which - OC_D_U];
      }
  return OC_OK;
}

/* Global error norms of the appendix accuracy test: the corner velocity
 * component `which` (OC_D_U, OC_D_V, OC_D_W) of level 1 of model a against
 * the finer model b at the corners the two grids share, over those corners of
 * a that lie above the height zmin (the grid points above the hill top):
 *   out[0] = L1 = (1/N) sum |psi_a - psi_b|,
 *   out[1] = L2 = ((1/N) sum (psi_a - psi_b)^2)^(1/2),   out[2] = N.
 * The spacings must be in one ratio dx_a / dx_b = p / q (integers, lowest
 * terms, q <= 16) in every direction over the same domain; corner I of a is
 * corner I p / q of b when q divides I, and only those corners count. */
int oc_error_norms(const oc_model *a, const oc_model *b, int which, double zmin, double *out) {
  if (which < OC_D_U || which > OC_D_W) return OC_EINVAL;
  int p = 0, q = 0;
  for (int qq = 1; qq <= 16 && !p; qq++) {
    double pp = a->P.dx / b->P.dx * qq;
    int pi = (int)floor(pp + 0.5);
    if (pi >= qq && fabs(pi - pp) <= 1e-9 * pp) { p = pi; q = qq; }
  }
  if (!p) return OC_EINVAL;
  if (fabs(p * b->P.dy - q * a->P.dy) > 1e-9 * q * a->P.dy || fabs(p * b->P.dz - q * a->P.dz) > 1e-9 * q * a->P.dz ||
      (long)a->nx * p != (long)b->nx * q || (long)a->ny * p != (long)b->ny * q || (long)a->nz * p != (long)b->nz * q)
    return OC_EINVAL;
  double s1 = 0.0, s2 = 0.0;
  long n = 0;
  for (int K = 0; K <= a->nz; K += q) {
    if (!(K * a->P.dz > zmin)) continue;
    for (int J = 0; J < a->ny; J += q)
      for (int I = 0; I < a->nx; I += q) {
        double ua[3], ub[3];
        corner_velocity(a, 1, I, J, K, ua);
        corner_velocity(b, 1, I / q * p, J / q * p, K / q * p, ub);
        double d = ua[which - OC_D_U] - ub[which - OC_D_U];
        s1 += fabs(d);
        s2 += d * d;
        n++;
      }
  }
  out[0] = n ? s1 / n : 0.0;
  out[1] = n ? sqrt(s2 / n) : 0.0;
  out[2] = (double)n;
  return OC_OK;
}

/* ================================================================== */
/* Block-structured refinement (Sec 2.2).                              */
/* Level 0 is the periodic domain with the lid; level l >= 1 is a box of */
/* nx_l x ny_l x nz_l cells of spacing 2^-l H that starts at the floor;  */
/* its cell i covers the cell (i + ox_l) / 2 of level l-1.               */
/* ================================================================== */
struct oc_refine {
  int nlev;
  oc_model *L[8];
  oc_box B[8]; /* B[l] for l >= 1 */
  /* flux register of the interface of level l+1 inside level l: the sums of
   * the fine face fluxes over the fine substeps, per coarse face */
  double *regm[8], *regh[8];
  long nsteps;
};

/* coarse cell of level l-1 covering fine cell (i,j,k) of level l */
static inline void parent(const oc_box *b, int i, int j, int k, int *ic, int *jc, int *kc) {
  *ic = (i + b->ox) >> 1; /* ox even and i + ox >= 0 */
  *jc = (j + b->oy) >> 1;
  *kc = k >> 1;
}

/* covered box of level l inside level l-1, in level l-1 cells */
static inline void covered(const oc_box *b, int *x0, int *x1, int *y0, int *y1, int *z1) {
  *x0 = b->ox / 2; *x1 = (b->ox + b->nx) / 2;
  *y0 = b->oy / 2; *y1 = (b->oy + b->ny) / 2;
  *z1 = b->nz / 2;
}

/* Coarse -> fine (Sec 2.2): at every exchange each fine ghost cell (all four
 * layers beyond the box) takes the value of the coarse cell that covers it
 * (injection), and each fine ghost corner outside the box's corners 0 .. n
 * (above nz at the top) the coarse momentum interpolated linearly along each
 * axis (coincident points copy; reading C-14).  Between exchanges the fine
 * level integrates the inner two ghost layers (cells -2 .. n+1, corners
 * -1 .. n+1) so that its boundary stencils see updated values; the exchange
 * then brings them back to the coarse solution.  All four time-level buffers
 * of the fine level receive the current coarse values. */
static void prolong(oc_model *c, oc_model *f, const oc_box *b) {
  for (int k = 0; k < f->nz + G; k++)
    for (int j = -G; j < f->ny + G; j++)
      for (int i = -G; i < f->nx + G; i++) {
        if (i >= 0 && i < f->nx && j >= 0 && j < f->ny && k < f->nz) continue;
        int ic, jc, kc;
        parent(b, i, j, k, &ic, &jc, &kc);
        long pc = CI(c, ic, jc, kc), pf = CI(f, i, j, k);
        for (int L = 0; L < 4; L++) {
          f->rp[L][pf] = c->rp[1][pc];
          f->pp[L][pf] = c->pp[1][pc];
        }
      }
  for (int K = -G + 1; K < f->nz + G; K++)
    for (int J = -G; J < f->ny + G; J++)
      for (int I = -G; I < f->nx + G; I++) {
        if (I >= 0 && I <= f->nx && J >= 0 && J <= f->ny && K <= f->nz) continue;
        int X = I + b->ox, Y = J + b->oy;
        int xs[2] = {X >> 1, (X + 1) >> 1}, ys[2] = {Y >> 1, (Y + 1) >> 1}, zs[2] = {K >> 1, (K + 1) >> 1};
        double s[3] = {0, 0, 0};
        for (int a = 0; a < 2; a++)
          for (int bb = 0; bb < 2; bb++)
            for (int cc = 0; cc < 2; cc++) {
              long pc = CI(c, xs[a], ys[bb], zs[cc]);
              s[0] += c->mx[1][pc]; s[1] += c->my[1][pc]; s[2] += c->mz[1][pc];
            }
        long pf = CI(f, I, J, K);
        for (int L = 0; L < 4; L++) {
          f->mx[L][pf] = s[0] / 8.0; f->my[L][pf] = s[1] / 8.0; f->mz[L][pf] = s[2] / 8.0;
        }
      }
}

/* Fine -> coarse (Sec 2.2): coarse cells of the covered box within G cells of
 * its boundary take the mean of the 8 fine cells they contain; coarse corners
 * inside the covered box or on its lateral and top faces (within G of them)
 * take the coincident fine corner (reading C-18: a corner on the interface is
 * covered by the fine level, so only one level computes it).  All four
 * time-level buffers of the coarse level receive the values. */
static void restrict_(oc_model *c, oc_model *f, const oc_box *b) {
  int x0, x1, y0, y1, z1;
  covered(b, &x0, &x1, &y0, &y1, &z1);
  for (int kc = 0; kc < z1; kc++)
    for (int jc = y0; jc < y1; jc++)
      for (int ic = x0; ic < x1; ic++) {
        int d = ic - x0;
        if (x1 - 1 - ic < d) d = x1 - 1 - ic;
        if (jc - y0 < d) d = jc - y0;
        if (y1 - 1 - jc < d) d = y1 - 1 - jc;
        if (z1 - 1 - kc < d) d = z1 - 1 - kc;
        if (d >= G) continue;
        double sr = 0, sp = 0;
        for (int dk = 0; dk < 2; dk++)
          for (int dj = 0; dj < 2; dj++)
            for (int di = 0; di < 2; di++) {
              long pf = CI(f, 2 * ic - b->ox + di, 2 * jc - b->oy + dj, 2 * kc + dk);
              sr += f->rp[1][pf];
              sp += f->pp[1][pf];
            }
        long pc = CI(c, ic, jc, kc);
        for (int L = 0; L < 4; L++) {
          c->rp[L][pc] = sr / 8.0;
          c->pp[L][pc] = sp / 8.0;
        }
      }
  for (int Kc = 1; Kc <= z1; Kc++)
    for (int Jc = y0; Jc <= y1; Jc++)
      for (int Ic = x0; Ic <= x1; Ic++) {
        int d = Ic - x0;
        if (x1 - Ic < d) d = x1 - Ic;
        if (Jc - y0 < d) d = Jc - y0;
        if (y1 - Jc < d) d = y1 - Jc;
        if (z1 - Kc < d) d = z1 - Kc;
        if (d > G) continue;
        long pf = CI(f, 2 * Ic - b->ox, 2 * Jc - b->oy, 2 * Kc), pc = CI(c, Ic, Jc, Kc);
        for (int L = 0; L < 4; L++) {
          c->mx[L][pc] = f->mx[1][pf]; c->my[L][pc] = f->my[1][pf]; c->mz[L][pc] = f->mz[1][pf];
        }
      }
}

/* coarse interface faces: the lateral faces of the covered box (x low,
 * x high, y low, y high) and its top, each with its first fine face */
typedef struct { int ax, I, J, K; int fi, fj, fk; } ifc;
static long interface_faces(const oc_box *b, ifc *out) {
  int x0, x1, y0, y1, z1;
  covered(b, &x0, &x1, &y0, &y1, &z1);
  long n = 0;
  for (int side = 0; side < 2; side++) {
    int Ic = side ? x1 : x0, If = side ? b->nx : 0;
    for (int kc = 0; kc < z1; kc++)
      for (int jc = y0; jc < y1; jc++) {
        if (out) { ifc f = {0, Ic, jc, kc, If, 2 * jc - b->oy, 2 * kc}; out[n] = f; }
        n++;
      }
  }
  for (int side = 0; side < 2; side++) {
    int Jc = side ? y1 : y0, Jf = side ? b->ny : 0;
    for (int kc = 0; kc < z1; kc++)
      for (int ic = x0; ic < x1; ic++) {
        if (out) { ifc f = {1, ic, Jc, kc, 2 * ic - b->ox, Jf, 2 * kc}; out[n] = f; }
        n++;
      }
  }
  for (int jc = y0; jc < y1; jc++)
    for (int ic = x0; ic < x1; ic++) {
      if (out) { ifc f = {2, ic, jc, z1, 2 * ic - b->ox, 2 * jc - b->oy, b->nz}; out[n] = f; }
      n++;
    }
  return n;
}

/* add the fine face fluxes of the last fine step to the register */
static void register_add(oc_refine *R, int l) {
  oc_model *f = R->L[l + 1];
  const oc_box *b = &R->B[l + 1];
  long n = interface_faces(b, NULL);
  ifc *F = (ifc *)xcalloc(n, sizeof(ifc));
  interface_faces(b, F);
  for (long q = 0; q < n; q++) {
    double sm = 0, sh = 0;
    for (int a = 0; a < 2; a++)
      for (int bb = 0; bb < 2; bb++) {
        long p;
        if (F[q].ax == 0) p = CI(f, F[q].fi, F[q].fj + a, F[q].fk + bb);
        else if (F[q].ax == 1) p = CI(f, F[q].fi + a, F[q].fj, F[q].fk + bb);
        else p = CI(f, F[q].fi + a, F[q].fj + bb, F[q].fk);
        const double *fm = F[q].ax == 0 ? f->fmx : (F[q].ax == 1 ? f->fmy : f->fmz);
        const double *fh = F[q].ax == 0 ? f->fhx : (F[q].ax == 1 ? f->fhy : f->fhz);
        sm += fm[p];
        sh += fh[p];
      }
    R->regm[l][q] += sm;
    R->regh[l][q] += sh;
  }
  free(F);
}

/* hand the register (mean over the two fine substeps; reading C-15) to the
 * coarse level, or withdraw it and clear the sums */
static void register_apply(oc_refine *R, int l, int on) {
  oc_model *c = R->L[l];
  const oc_box *b = &R->B[l + 1];
  long n = interface_faces(b, NULL);
  ifc *F = (ifc *)xcalloc(n, sizeof(ifc));
  interface_faces(b, F);
  for (long q = 0; q < n; q++) {
    long p = CI(c, F[q].I, F[q].J, F[q].K);
    int8_t *ov = F[q].ax == 0 ? c->ovx : (F[q].ax == 1 ? c->ovy : c->ovz);
    double *om = F[q].ax == 0 ? c->ovmx : (F[q].ax == 1 ? c->ovmy : c->ovmz);
    double *oh = F[q].ax == 0 ? c->ovhx : (F[q].ax == 1 ? c->ovhy : c->ovhz);
    ov[p] = (int8_t)on;
    om[p] = 0.5 * R->regm[l][q];
    oh[p] = 0.5 * R->regh[l][q];
    if (!on) { R->regm[l][q] = 0.0; R->regh[l][q] = 0.0; }
  }
  free(F);
}

/* cycle(l): the finer level first, two steps, then this level, then the
 * exchange with the finer level (Sec 2.2) */
static void cycle(oc_refine *R, int l) {
  if (l + 1 < R->nlev) {
    for (int s = 0; s < 2; s++) {
      cycle(R, l + 1);
      register_add(R, l);
    }
    register_apply(R, l, 1);
  }
  oc_step(R->L[l], 1);
  if (l + 1 < R->nlev) {
    register_apply(R, l, 0);
    restrict_(R->L[l], R->L[l + 1], &R->B[l + 1]);
    prolong(R->L[l], R->L[l + 1], &R->B[l + 1]);
  }
}

void oc_refine_destroy(oc_refine *R) {
  if (!R) return;
  for (int l = 0; l < R->nlev; l++) {
    oc_destroy(R->L[l]);
    free(R->regm[l]);
    free(R->regh[l]);
  }
  free(R);
}

oc_refine *oc_refine_create(const oc_params *P0, int nlev, const oc_box *boxes, const double *h_finest,
                            int *status) {
  *status = OC_EINVAL;
  if (nlev < 1 || nlev > 8) return NULL;
  oc_refine *R = (oc_refine *)calloc(1, sizeof(oc_refine));
  R->nlev = nlev;
  for (int l = 0; l < nlev; l++) {
    oc_params P = *P0;
    double f = ldexp(1.0, -l);
    P.dx = P0->dx * f; P.dy = P0->dy * f; P.dz = P0->dz * f; P.dt = P0->dt * f;
    P.ztop = P0->nz * P0->dz;
    if (l > 0) {
      R->B[l] = boxes[l - 1];
      const oc_box *b = &R->B[l];
      const oc_model *c = R->L[l - 1];
      int x0, x1, y0, y1, z1;
      covered(b, &x0, &x1, &y0, &y1, &z1);
      /* even extents and offsets, and at least 8 coarse cells between the
       * covered box and the coarser level's edges and top */
      int bad = ((b->ox | b->oy | b->nx | b->ny | b->nz) & 1) || x0 < 8 || y0 < 8 ||
                x1 > c->nx - 8 || y1 > c->ny - 8 || z1 > c->nz - 8;
      if (bad) {
        oc_refine_destroy(R);
        return NULL;
      }
      P.nx = b->nx; P.ny = b->ny; P.nz = b->nz;
    }
    int finest = (l == nlev - 1);
    long nh = l == 0 ? (long)P.nx * P.ny : (long)(P.nx + 2 * G + 1) * (P.ny + 2 * G + 1);
    double *h = (double *)xcalloc(nh, sizeof(double));
    if (finest && h_finest) memcpy(h, h_finest, sizeof(double) * nh);
    int st;
    R->L[l] = level_create(&P, l == 0, l == 0, h, &st);
    free(h);
    if (!R->L[l]) {
      *status = st;
      oc_refine_destroy(R);
      return NULL;
    }
    if (l > 0) {
      long n = interface_faces(&R->B[l], NULL);
      R->regm[l - 1] = xcalloc(n, 8);
      R->regh[l - 1] = xcalloc(n, 8);
    }
  }
  *status = OC_OK;
  return R;
}

void oc_refine_init(oc_refine *R) {
  for (int l = 0; l < R->nlev; l++) oc_init_state(R->L[l]);
  for (int l = 0; l + 1 < R->nlev; l++) {
    restrict_(R->L[l], R->L[l + 1], &R->B[l + 1]);
    prolong(R->L[l], R->L[l + 1], &R->B[l + 1]);
  }
  R->nsteps = 0;
}

void oc_refine_step(oc_refine *R, int n) {
  for (int s = 0; s < n; s++) {
    cycle(R, 0);
    R->nsteps++;
  }
}

oc_model *oc_refine_level(oc_refine *R, int l) { return (l >= 0 && l < R->nlev) ? R->L[l] : NULL; }

/* Two-level perturbation mass over the active cells of every level:
 * sum V (rho'(n) + rho'(n-1)), covered cells excluded (the invariant of the
 * leapfrog with the flux register when the filter is off; reading C-15). */
double oc_refine_mass(oc_refine *R, int both) {
  double s = 0.0;
  for (int l = 0; l < R->nlev; l++) {
    oc_model *m = R->L[l];
    int x0 = 0, x1 = 0, y0 = 0, y1 = 0, z1 = 0, has = l + 1 < R->nlev;
    if (has) covered(&R->B[l + 1], &x0, &x1, &y0, &y1, &z1);
    for (int k = 0; k < m->nz; k++)
      for (int j = 0; j < m->ny; j++)
        for (int i = 0; i < m->nx; i++) {
          if (has && i >= x0 && i < x1 && j >= y0 && j < y1 && k < z1) continue;
          long c = CI(m, i, j, k);
          if (m->cls[c] != C_UG && m->root[c] == c)
            s += m->vg[c] * (m->rp[1][c] + (both ? m->rp[0][c] : 0.0));
        }
  }
  return s;
}
