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
 *   Sec 2.2  leapfrog with the Robert-Asselin filter.
 *
 * Readings of points the paper leaves open are listed in the design notes
 * and in the comments at the place they apply ("reading:").
 *
 * Volumes and apertures use exact integration of the bilinear surface
 * (closed form along every vertical face, piecewise Gauss-Legendre over
 * smooth x-segments inside a column), exact for planar terrain.
 *
 * Parity pins: see tests/test_oracle_*.py.  Every function here is pinned
 * by at least one test against a closed form, a brute-force computation or
 * an invariant the paper states.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "oracle.h"

#define GZ 2 /* corner levels kept below the floor and above the lid */

enum { C_UG = 0, C_FULL = 1, C_CUT = 2, C_ABS = 3 };    /* cell classes   */
enum { V_UG = 0, V_PRED = 1, V_MF = 2, V_LID = 3 };     /* corner classes */

struct oc_model {
  oc_params P;
  int nx, ny, nz;
  long ncell, ncol, ncorner, nzface;
  /* geometry */
  double *h;          /* corner heights, nx*ny (periodic)              */
  double *hc, *gx, *gy; /* column centre height and gradients, nx*ny   */
  double *vf;         /* volume fraction V/V0 per cell                 */
  double *ax, *ay;    /* lateral face apertures: ax at (I,j,k) is the face x=I*dx */
  double *az;         /* horizontal face apertures, (nz+1) levels      */
  int8_t *cls;        /* cell class                                    */
  int32_t *target;    /* merge target cell (absorbed cells), else -1   */
  int32_t *root;      /* representative (host) cell of the merge group */
  double *vg;         /* group volume at the host                      */
  long *gstart, *gmem;  /* members of the group of host r: gmem[gstart[r] .. gstart[r+1]) */
  int8_t *vcls;       /* corner class, levels -GZ..nz+GZ               */
  int32_t *bK, *bI, *bJ; double *ba, *bb, *bn; /* boundary-point stencil */
  int32_t *mK; double *mg;                     /* merged-face stencil   */
  /* base state, levels -GZ-2 .. nz+GZ+2 */
  double *rhob, *pb, *thb; int boff, nb;
  double *rhobc, *tau; /* corner levels -GZ..nz+GZ */
  /* state: 0 = old (filtered n-1), 1 = current n, 2 = new n+1, 3 = filtered n */
  double *rp[4], *pp[4], *mx[4], *my[4], *mz[4];
  double *ub[4];      /* boundary-point velocity (3 per column) per level */
  /* work */
  double *rho_t, *th_t, *thp_o, *rhoc, *vel, *RM, *RH;
  int nsteps;
};

/* ------------------------------------------------------------------ */
/* indexing                                                           */
static inline int wrap(int i, int n) { int r = i % n; return r < 0 ? r + n : r; }
static inline long CI(const oc_model *m, int i, int j, int k) {
  return ((long)k * m->ny + wrap(j, m->ny)) * m->nx + wrap(i, m->nx);
}
static inline long QI(const oc_model *m, int i, int j) {
  return (long)wrap(j, m->ny) * m->nx + wrap(i, m->nx);
}
/* corners: levels K in [-GZ, nz+GZ] */
static inline long PI_(const oc_model *m, int I, int J, int K) {
  return ((long)(K + GZ) * m->ny + wrap(J, m->ny)) * m->nx + wrap(I, m->nx);
}
static inline long ZF(const oc_model *m, int i, int j, int K) {
  return ((long)K * m->ny + wrap(j, m->ny)) * m->nx + wrap(i, m->nx);
}
static inline double HC(const oc_model *m, int I, int J) { return m->h[QI(m, I, J)]; }

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
  double **dp[] = {&m->h, &m->hc, &m->gx, &m->gy, &m->vf, &m->ax, &m->ay, &m->az, &m->vg,
                   &m->ba, &m->bb, &m->bn, &m->mg, &m->rhob, &m->pb, &m->thb, &m->rhobc,
                   &m->tau, &m->rho_t, &m->th_t, &m->thp_o, &m->rhoc, &m->vel, &m->RM, &m->RH};
  for (size_t i = 0; i < sizeof(dp) / sizeof(dp[0]); i++) free(*dp[i]);
  free(m->gstart); free(m->gmem);
  free(m->cls); free(m->target); free(m->root); free(m->vcls);
  free(m->bK); free(m->bI); free(m->bJ); free(m->mK);
  for (int l = 0; l < 4; l++) {
    free(m->rp[l]); free(m->pp[l]); free(m->mx[l]); free(m->my[l]); free(m->mz[l]); free(m->ub[l]);
  }
  free(m);
}

static int build_geometry(oc_model *m);

oc_model *oc_create(const oc_params *P, const double *h, int *status) {
  *status = OC_EINVAL;
  if (P->nx < 4 || P->ny < 4 || P->nz < 4) return NULL;
  oc_model *m = (oc_model *)calloc(1, sizeof(oc_model));
  m->P = *P;
  m->nx = P->nx; m->ny = P->ny; m->nz = P->nz;
  m->ncol = (long)m->nx * m->ny;
  m->ncell = m->ncol * m->nz;
  m->ncorner = m->ncol * (m->nz + 1 + 2 * GZ);
  m->nzface = m->ncol * (m->nz + 1);
  m->h = xcalloc(m->ncol, sizeof(double));
  memcpy(m->h, h, sizeof(double) * m->ncol);
  m->hc = xcalloc(m->ncol, 8); m->gx = xcalloc(m->ncol, 8); m->gy = xcalloc(m->ncol, 8);
  m->vf = xcalloc(m->ncell, 8); m->ax = xcalloc(m->ncell, 8); m->ay = xcalloc(m->ncell, 8);
  m->az = xcalloc(m->nzface, 8);
  m->cls = xcalloc(m->ncell, 1); m->target = xcalloc(m->ncell, 4); m->root = xcalloc(m->ncell, 4);
  m->vg = xcalloc(m->ncell, 8);
  m->gstart = xcalloc(m->ncell + 1, sizeof(long)); m->gmem = xcalloc(m->ncell, sizeof(long));
  m->vcls = xcalloc(m->ncorner, 1);
  m->bK = xcalloc(m->ncol, 4); m->bI = xcalloc(m->ncol, 4); m->bJ = xcalloc(m->ncol, 4);
  m->ba = xcalloc(m->ncol, 8); m->bb = xcalloc(m->ncol, 8); m->bn = xcalloc(3 * m->ncol, 8);
  m->mK = xcalloc(m->ncorner, 4); m->mg = xcalloc(m->ncorner, 8);
  /* base state at cell levels k in [-GZ-2, nz+GZ+2) */
  m->boff = GZ + 2;
  m->nb = m->nz + 2 * (GZ + 2);
  m->rhob = xcalloc(m->nb, 8); m->pb = xcalloc(m->nb, 8); m->thb = xcalloc(m->nb, 8);
  for (int kk = 0; kk < m->nb; kk++) {
    int k = kk - m->boff;
    base_state(P, (k + 0.5) * P->dz, &m->rhob[kk], &m->pb[kk]);
    m->thb[kk] = rhotheta_of_p(P, m->pb[kk]);
  }
  int nzc = m->nz + 1 + 2 * GZ;
  m->rhobc = xcalloc(nzc, 8); m->tau = xcalloc(nzc, 8);
  double ztop = m->nz * P->dz, zs = ztop * (1.0 - P->sponge_frac);
  for (int KK = 0; KK < nzc; KK++) {
    int K = KK - GZ;
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
    m->rp[l] = xcalloc(m->ncell, 8); m->pp[l] = xcalloc(m->ncell, 8);
    m->mx[l] = xcalloc(m->ncorner, 8); m->my[l] = xcalloc(m->ncorner, 8);
    m->mz[l] = xcalloc(m->ncorner, 8);
    m->ub[l] = xcalloc(3 * m->ncol, 8);
  }
  m->rho_t = xcalloc(m->ncell, 8); m->th_t = xcalloc(m->ncell, 8); m->thp_o = xcalloc(m->ncell, 8);
  m->rhoc = xcalloc(m->ncorner, 8); m->vel = xcalloc(3 * m->ncorner, 8);
  m->RM = xcalloc(m->ncell, 8); m->RH = xcalloc(m->ncell, 8);
  int st = build_geometry(m);
  *status = st;
  if (st != OC_OK) { oc_destroy(m); return NULL; }
  return m;
}

/* ------------------------------------------------------------------ */
static int build_geometry(oc_model *m) {
  const oc_params *P = &m->P;
  int nx = m->nx, ny = m->ny, nz = m->nz;
  double dx = P->dx, dy = P->dy, dz = P->dz;

  /* column centre height (bilinear value at the centre = mean of corners) and
   * the column gradients of Eqs. xgrad / ygrad */
  for (int j = 0; j < ny; j++)
    for (int i = 0; i < nx; i++) {
      double h00 = HC(m, i, j), h10 = HC(m, i + 1, j), h01 = HC(m, i, j + 1), h11 = HC(m, i + 1, j + 1);
      long q = QI(m, i, j);
      m->hc[q] = 0.25 * (h00 + h10 + h01 + h11);
      m->gx[q] = ((h10 + h11) - (h00 + h01)) / (2.0 * dx);
      m->gy[q] = ((h01 + h11) - (h00 + h10)) / (2.0 * dy);
    }

  /* volumes and classes */
  for (int k = 0; k < nz; k++)
    for (int j = 0; j < ny; j++)
      for (int i = 0; i < nx; i++) {
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
  for (int k = 0; k < nz; k++)
    for (int j = 0; j < ny; j++)
      for (int I = 0; I < nx; I++) {
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
        m->ay[CI(m, I, j, k)] = a; /* face y = j*dy of cell (I, j, k) */
      }
  /* horizontal apertures; the floor (K=0) and the rigid lid (K=nz) are walls */
  for (int K = 0; K <= nz; K++)
    for (int j = 0; j < ny; j++)
      for (int i = 0; i < nx; i++) {
        double a = 0.0;
        if (K > 0 && K < nz) {
          double z = K * dz;
          double h00 = HC(m, i, j), h10 = HC(m, i + 1, j), h01 = HC(m, i, j + 1), h11 = HC(m, i + 1, j + 1);
          double hmin = fmin(fmin(h00, h10), fmin(h01, h11));
          double hmax = fmax(fmax(h00, h10), fmax(h01, h11));
          if (z > hmax) a = 1.0;
          else if (z <= hmin) a = 0.0;
          else a = oc_col_int(z, h00, h10, h01, h11, dx, dy, 1) / (dx * dy);
        }
        m->az[ZF(m, i, j, K)] = a;
      }

  /* merge direction, Fig. 6 pseudocode */
  for (int k = 0; k < nz; k++)
    for (int j = 0; j < ny; j++)
      for (int i = 0; i < nx; i++) {
        long c = CI(m, i, j, k);
        if (m->cls[c] != C_ABS) continue;
        double gx = m->gx[QI(m, i, j)], gy = m->gy[QI(m, i, j)];
        double agx = fabs(gx), agy = fabs(gy);
        long t;
        if (agx <= 1.0 && agy <= 1.0) {
          if (k + 1 >= nz) return OC_EGEOM;
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
        m->target[c] = (int32_t)t;
      }
  /* merge groups: follow targets to the representative (host) cell; a chain
   * that ends underground or loops is a geometry failure ("v-shaped valley") */
  for (long c = 0; c < m->ncell; c++) {
    if (m->cls[c] == C_UG) { m->root[c] = -1; continue; }
    long r = c;
    int n = 0;
    while (m->cls[r] == C_ABS) {
      r = m->target[r];
      if (++n > 64) return OC_EGEOM;
    }
    if (m->cls[r] == C_UG) return OC_EGEOM;
    m->root[c] = (int32_t)r;
  }
  /* members of each group in ascending cell order, and the group volume */
  for (long c = 0; c <= m->ncell; c++) m->gstart[c] = 0;
  for (long c = 0; c < m->ncell; c++)
    if (m->root[c] >= 0) m->gstart[m->root[c] + 1]++;
  for (long c = 0; c < m->ncell; c++) m->gstart[c + 1] += m->gstart[c];
  {
    long *fill = (long *)xcalloc(m->ncell, sizeof(long));
    for (long c = 0; c < m->ncell; c++)
      if (m->root[c] >= 0) {
        long r = m->root[c];
        m->gmem[m->gstart[r] + fill[r]++] = c;
      }
    free(fill);
  }
  for (long r = 0; r < m->ncell; r++) {
    double v = 0.0;
    for (long a = m->gstart[r]; a < m->gstart[r + 1]; a++) v += m->vf[m->gmem[a]] * dx * dy * dz;
    m->vg[r] = v;
  }

  /* velocity-point classes on corners, Sec 2.3 / Fig. 7 and Sec 2.4 */
  for (int K = -GZ; K <= nz + GZ; K++)
    for (int J = 0; J < ny; J++)
      for (int I = 0; I < nx; I++) {
        long p = PI_(m, I, J, K);
        int8_t v;
        if (K * dz <= HC(m, I, J)) v = V_UG;
        else if (K >= nz) v = V_LID;
        else if (K < 1) v = V_MF;
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
  for (int J = 0; J < ny; J++)
    for (int I = 0; I < nx; I++)
      if (m->vcls[PI_(m, I, J, nz - 1)] != V_PRED) return OC_EGEOM;

  /* boundary-point stencils: unit normal from the corner gradients of the
   * column-centre heights, then the nearest plane of four predicted points
   * crossed by the normal line (Sec 2.4, nearest-plane construction) */
  for (int J = 0; J < ny; J++)
    for (int I = 0; I < nx; I++) {
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
      for (int K = K0; K < K0 + 8 && K <= nz - 1; K++) {
        double t = (K * dz - hh) / nzv;
        double xN = I * dx + t * nxv, yN = J * dy + t * nyv;
        double fi = floor(xN / dx), fj = floor(yN / dy);
        int i0 = (int)fi, j0 = (int)fj;
        double a = xN / dx - fi, b = yN / dy - fj;
        /* every point of the plane that carries a nonzero bilinear weight must
         * be a predicted point (on a grid line only that line is needed) */
        int ok = m->vcls[PI_(m, i0, j0, K)] == V_PRED &&
                 (a == 0.0 || m->vcls[PI_(m, i0 + 1, j0, K)] == V_PRED) &&
                 (b == 0.0 || m->vcls[PI_(m, i0, j0 + 1, K)] == V_PRED) &&
                 (a == 0.0 || b == 0.0 || m->vcls[PI_(m, i0 + 1, j0 + 1, K)] == V_PRED);
        if (ok) {
          m->bK[q] = K; m->bI[q] = wrap(i0, nx); m->bJ[q] = wrap(j0, ny);
          m->ba[q] = a; m->bb[q] = b;
          found = 1;
          break;
        }
      }
      if (!found) return OC_EGEOM;
    }
  /* merged-face points: interpolate along the vertical line between the
   * boundary point and the nearest predicted point above */
  for (int K = 0; K <= nz; K++)
    for (int J = 0; J < ny; J++)
      for (int I = 0; I < nx; I++) {
        long p = PI_(m, I, J, K);
        m->mK[p] = -1; m->mg[p] = 0.0;
        if (m->vcls[p] != V_MF) continue;
        int ka = -1;
        for (int K2 = K + 1; K2 <= nz - 1; K2++)
          if (m->vcls[PI_(m, I, J, K2)] == V_PRED) { ka = K2; break; }
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
  if (k < 0 || k >= m->nz) return rhob_k(m, k);
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
 * vertical line; every other corner holds momentum / corner density. */
static void corner_velocity(const oc_model *m, int L, int I, int J, int K, double u[3]) {
  if (K * m->P.dz <= HC(m, I, J)) {
    long q = QI(m, I, J);
    u[0] = m->ub[L][3 * q]; u[1] = m->ub[L][3 * q + 1]; u[2] = m->ub[L][3 * q + 2];
    return;
  }
  long p = PI_(m, I, J, K);
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
  int nx = m->nx, ny = m->ny, nz = m->nz;
  double dz = m->P.dz;
  for (int J = 0; J < ny; J++)
    for (int I = 0; I < nx; I++) {
      long q = QI(m, I, J);
      double uN[3] = {0, 0, 0};
      int K = m->bK[q], i0 = m->bI[q], j0 = m->bJ[q];
      double a = m->ba[q], b = m->bb[q];
      double w[4] = {(1 - a) * (1 - b), a * (1 - b), (1 - a) * b, a * b};
      int ci[4] = {i0, i0 + 1, i0, i0 + 1}, cj[4] = {j0, j0, j0 + 1, j0 + 1};
      for (int s = 0; s < 4; s++) {
        double u[3];
        long p = PI_(m, ci[s], cj[s], K);
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
  for (int J = 0; J < ny; J++)
    for (int I = 0; I < nx; I++) {
      long q = QI(m, I, J);
      double hh = HC(m, I, J);
      for (int K = -GZ; K <= nz + GZ; K++) {
        long p = PI_(m, I, J, K);
        int v = m->vcls[p];
        double u[3];
        if (v == V_PRED) continue;
        if (v == V_UG) {
          for (int d = 0; d < 3; d++) u[d] = m->ub[L][3 * q + d];
        } else if (v == V_LID) {
          double ul[3];
          long pl = PI_(m, I, J, nz - 1);
          double rl = rho_corner(m, L, I, J, nz - 1);
          ul[0] = m->mx[L][pl] / rl; ul[1] = m->my[L][pl] / rl;
          u[0] = ul[0]; u[1] = ul[1]; u[2] = 0.0;
        } else { /* merged face */
          int ka = m->mK[p];
          double g = m->mg[p];
          long pa = PI_(m, I, J, ka);
          double ra = rho_corner(m, L, I, J, ka);
          double ua[3] = {m->mx[L][pa] / ra, m->my[L][pa] / ra, m->mz[L][pa] / ra};
          for (int d = 0; d < 3; d++) u[d] = g * ua[d] + (1.0 - g) * m->ub[L][3 * q + d];
        }
        (void)hh;
        double rc = rho_corner(m, L, I, J, K);
        m->mx[L][p] = rc * u[0]; m->my[L][p] = rc * u[1]; m->mz[L][p] = rc * u[2];
      }
    }
}

/* ------------------------------------------------------------------ */
void oc_init_state(oc_model *m) {
  const oc_params *P = &m->P;
  for (int l = 0; l < 4; l++) {
    memset(m->rp[l], 0, sizeof(double) * m->ncell);
    memset(m->pp[l], 0, sizeof(double) * m->ncell);
    memset(m->mx[l], 0, sizeof(double) * m->ncorner);
    memset(m->my[l], 0, sizeof(double) * m->ncorner);
    memset(m->mz[l], 0, sizeof(double) * m->ncorner);
    memset(m->ub[l], 0, sizeof(double) * 3 * m->ncol);
  }
  /* uniform flow U on predicted points; zero perturbations */
  for (int K = -GZ; K <= m->nz + GZ; K++)
    for (int J = 0; J < m->ny; J++)
      for (int I = 0; I < m->nx; I++) {
        long p = PI_(m, I, J, K);
        if (m->vcls[p] == V_PRED) m->mx[1][p] = rho_corner(m, 1, I, J, K) * P->U;
      }
  diagnose_velocity(m, 1);
  m->nsteps = 0;
}

/* ------------------------------------------------------------------ */
/* One leapfrog step.  Level 0 = filtered n-1, 1 = n; writes 2 = n+1 and
 * 3 = filtered n, then rotates so that (0,1) = (filtered n, n+1).
 * The first step is forward Euler: old = current, half the leapfrog interval,
 * no filter (reading C-3). */
static void scalar_residuals(oc_model *m);

void oc_step(oc_model *m, int nsteps) {
  const oc_params *P = &m->P;
  int nx = m->nx, ny = m->ny, nz = m->nz;
  double dx = P->dx, dy = P->dy, dz = P->dz, V0 = dx * dy * dz;
  double kap = P->R / P->cp, Cp = P->cp * P->R / (P->cp - P->R);
  for (int s = 0; s < nsteps; s++) {
    int first = (m->nsteps == 0);
    int O = first ? 1 : 0; /* level used as "n-1" */
    double dt2 = first ? P->dt : 2.0 * P->dt;
    double nu = first ? 0.0 : P->ra_nu;
    double kdif = P->c4 / (16.0 * P->dt);

    /* cell totals at n and the rho-theta perturbation at n-1 */
    for (int k = 0; k < nz; k++)
      for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
          long c = CI(m, i, j, k);
          m->rho_t[c] = rhob_k(m, k) + m->rp[1][c];
          m->th_t[c] = rhotheta_of_p(P, pb_k(m, k) + m->pp[1][c]);
          m->thp_o[c] = rhotheta_of_p(P, pb_k(m, k) + m->pp[O][c]) - thb_k(m, k);
        }
    /* corner velocities at n */
    for (int K = -GZ; K <= nz + GZ; K++)
      for (int J = 0; J < ny; J++)
        for (int I = 0; I < nx; I++) {
          long p = PI_(m, I, J, K);
          corner_velocity(m, 1, I, J, K, &m->vel[3 * p]);
        }
    scalar_residuals(m);

    /* scalar update per merge group (Sec 2.3/2.4): divergence over the
     * merged volume, host update, scatter to the absorbed cells */
    for (long c = 0; c < m->ncell; c++) {
      m->rp[2][c] = 0.0; m->pp[2][c] = 0.0; m->rp[3][c] = 0.0; m->pp[3][c] = 0.0;
    }
    for (long r = 0; r < m->ncell; r++) {
      if (m->cls[r] == C_UG || m->root[r] != r) continue;
      double rm = 0.0, rh = 0.0;
      for (long a = m->gstart[r]; a < m->gstart[r + 1]; a++) {
        rm += m->RM[m->gmem[a]]; rh += m->RH[m->gmem[a]];
      }
      double VG = m->vg[r];
      int kr = (int)(r / m->ncol), jr = (int)((r / nx) % ny), ir = (int)(r % nx);
      /* fourth-order artificial diffusion of (rho theta)' at n-1 (reading C-4) */
      double d4 = 0.0;
      {
        double f[5];
        for (int a = -2; a <= 2; a++) f[a + 2] = m->thp_o[CI(m, ir + a, jr, kr)];
        d4 += f[0] - 4 * f[1] + 6 * f[2] - 4 * f[3] + f[4];
        for (int a = -2; a <= 2; a++) f[a + 2] = m->thp_o[CI(m, ir, jr + a, kr)];
        d4 += f[0] - 4 * f[1] + 6 * f[2] - 4 * f[3] + f[4];
        for (int a = -2; a <= 2; a++) {
          int kk = kr + a;
          f[a + 2] = (kk < 0 || kk >= nz) ? 0.0 : m->thp_o[CI(m, ir, jr, kk)];
        }
        d4 += f[0] - 4 * f[1] + 6 * f[2] - 4 * f[3] + f[4];
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
    for (int K = -GZ; K <= nz + GZ; K++)
      for (int J = 0; J < ny; J++)
        for (int I = 0; I < nx; I++) {
          long p = PI_(m, I, J, K);
          if (m->vcls[p] != V_PRED) continue;
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
          const double *uE = &m->vel[3 * PI_(m, I + 1, J, K)], *uW = &m->vel[3 * PI_(m, I - 1, J, K)];
          const double *uN = &m->vel[3 * PI_(m, I, J + 1, K)], *uS = &m->vel[3 * PI_(m, I, J - 1, K)];
          const double *uT = &m->vel[3 * PI_(m, I, J, K + 1)], *uB = &m->vel[3 * PI_(m, I, J, K - 1)];
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
          for (int d = 0; d < 3; d++) {
            /* reference momentum (rho_bar_corner U, 0, 0) at corner level K */
            double ref0 = d == 0 ? m->rhobc[K + GZ] * P->U : 0.0;
            double f[5], d4 = 0.0;
            for (int a = -2; a <= 2; a++) f[a + 2] = MO[d][PI_(m, I + a, J, K)] - ref0;
            d4 += f[0] - 4 * f[1] + 6 * f[2] - 4 * f[3] + f[4];
            for (int a = -2; a <= 2; a++) f[a + 2] = MO[d][PI_(m, I, J + a, K)] - ref0;
            d4 += f[0] - 4 * f[1] + 6 * f[2] - 4 * f[3] + f[4];
            for (int a = -2; a <= 2; a++)
              f[a + 2] = MO[d][PI_(m, I, J, K + a)] - (d == 0 ? m->rhobc[K + a + GZ] * P->U : 0.0);
            d4 += f[0] - 4 * f[1] + 6 * f[2] - 4 * f[3] + f[4];
            tend[d] += -kdif * d4 - m->tau[K + GZ] * (MO[d][p] - ref0);
          }
          double *MN[3] = {m->mx[2], m->my[2], m->mz[2]};
          for (int d = 0; d < 3; d++) MN[d][p] = MO[d][p] + dt2 * tend[d];
        }
    /* steps 2 and 3 of the velocity calculation on the new level; they need
     * the new densities, so they follow the scalar update */
    diagnose_velocity(m, 2);
    /* Robert-Asselin filter on every corner value (prognostic or diagnosed) */
    for (long p = 0; p < m->ncorner; p++) {
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
 * faces inside one merge group are skipped (they cancel in the group sum). */
static void scalar_residuals(oc_model *m) {
  const oc_params *P = &m->P;
  int nx = m->nx, ny = m->ny, nz = m->nz;
  double dx = P->dx, dy = P->dy, dz = P->dz;
  for (int k = 0; k < nz; k++)
    for (int j = 0; j < ny; j++)
      for (int i = 0; i < nx; i++) {
        long c = CI(m, i, j, k);
        m->RM[c] = 0.0; m->RH[c] = 0.0;
        if (m->cls[c] == C_UG) continue;
        double rm = 0.0, rh = 0.0;
        /* six faces: (axis, side) with side +1 = high face */
        for (int ax = 0; ax < 3; ax++)
          for (int sd = 0; sd <= 1; sd++) {
            int ni = i, nj = j, nk = k;
            double A, S;
            int cI[4], cJ[4], cK[4];
            if (ax == 0) {
              int I = i + sd;
              ni = i + (sd ? 1 : -1);
              A = m->ax[CI(m, I, j, k)];
              S = dy * dz;
              int cc[4][3] = {{I, j, k}, {I, j + 1, k}, {I, j, k + 1}, {I, j + 1, k + 1}};
              for (int s = 0; s < 4; s++) { cI[s] = cc[s][0]; cJ[s] = cc[s][1]; cK[s] = cc[s][2]; }
            } else if (ax == 1) {
              int J = j + sd;
              nj = j + (sd ? 1 : -1);
              A = m->ay[CI(m, i, J, k)];
              S = dx * dz;
              int cc[4][3] = {{i, J, k}, {i + 1, J, k}, {i, J, k + 1}, {i + 1, J, k + 1}};
              for (int s = 0; s < 4; s++) { cI[s] = cc[s][0]; cJ[s] = cc[s][1]; cK[s] = cc[s][2]; }
            } else {
              int K = k + sd;
              nk = k + (sd ? 1 : -1);
              A = m->az[ZF(m, i, j, K)];
              S = dx * dy;
              int cc[4][3] = {{i, j, K}, {i + 1, j, K}, {i, j + 1, K}, {i + 1, j + 1, K}};
              for (int s = 0; s < 4; s++) { cI[s] = cc[s][0]; cJ[s] = cc[s][1]; cK[s] = cc[s][2]; }
            }
            if (A == 0.0) continue;
            if (nk < 0 || nk >= nz) continue;
            long nc = CI(m, ni, nj, nk);
            if (m->cls[nc] != C_UG && m->root[nc] == m->root[c]) continue;
            double un = 0.0;
            for (int s = 0; s < 4; s++) un += m->vel[3 * PI_(m, cI[s], cJ[s], cK[s]) + ax];
            un *= 0.25;
            double fm = 0.5 * (m->rho_t[c] + m->rho_t[nc]) * un * A * S;
            double fh = 0.5 * (m->th_t[c] + m->th_t[nc]) * un * A * S;
            if (sd) { rm += fm; rh += fh; } else { rm -= fm; rh -= fh; }
          }
        m->RM[c] = rm; m->RH[c] = rh;
      }
}

/* ------------------------------------------------------------------ */
/* accessors */
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
  *ncell = m->ncell; *ncorner = m->ncorner; *ncol = m->ncol; *gz = GZ;
  return OC_OK;
}

int oc_get_state(oc_model *m, int field, int level, double *out) {
  if (level < 0 || level > 1) return OC_EINVAL;
  double *a = level_array(m, field, level);
  if (!a) return OC_EINVAL;
  long n = (field == OC_F_RHOP || field == OC_F_PP) ? m->ncell : (field == OC_F_UB ? 3 * m->ncol : m->ncorner);
  memcpy(out, a, sizeof(double) * n);
  return OC_OK;
}

int oc_set_state(oc_model *m, int field, int level, const double *in) {
  if (level < 0 || level > 1) return OC_EINVAL;
  double *a = level_array(m, field, level);
  if (!a) return OC_EINVAL;
  long n = (field == OC_F_RHOP || field == OC_F_PP) ? m->ncell : (field == OC_F_UB ? 3 * m->ncol : m->ncorner);
  memcpy(a, in, sizeof(double) * n);
  return OC_OK;
}

int oc_get_geometry(const oc_model *m, double *vf, double *ax, double *ay, double *az, int8_t *cls,
                    int32_t *root, double *vg, double *hc, double *gx, double *gy) {
  memcpy(vf, m->vf, 8 * m->ncell); memcpy(ax, m->ax, 8 * m->ncell); memcpy(ay, m->ay, 8 * m->ncell);
  memcpy(az, m->az, 8 * m->nzface); memcpy(cls, m->cls, m->ncell); memcpy(root, m->root, 4 * m->ncell);
  memcpy(vg, m->vg, 8 * m->ncell);
  memcpy(hc, m->hc, 8 * m->ncol); memcpy(gx, m->gx, 8 * m->ncol); memcpy(gy, m->gy, 8 * m->ncol);
  return OC_OK;
}

int oc_get_points(const oc_model *m, int8_t *vcls, int32_t *bK, int32_t *bI, int32_t *bJ, double *ba,
                  double *bb, double *bn, int32_t *mK, double *mg) {
  memcpy(vcls, m->vcls, m->ncorner);
  memcpy(bK, m->bK, 4 * m->ncol); memcpy(bI, m->bI, 4 * m->ncol); memcpy(bJ, m->bJ, 4 * m->ncol);
  memcpy(ba, m->ba, 8 * m->ncol); memcpy(bb, m->bb, 8 * m->ncol); memcpy(bn, m->bn, 24 * m->ncol);
  memcpy(mK, m->mK, 4 * m->ncorner); memcpy(mg, m->mg, 8 * m->ncorner);
  return OC_OK;
}

int oc_get_base(const oc_model *m, double *rhob, double *pb, int *koff, int *nb) {
  memcpy(rhob, m->rhob, 8 * m->nb); memcpy(pb, m->pb, 8 * m->nb);
  *koff = m->boff; *nb = m->nb;
  return OC_OK;
}

/* Perturbation mass: sum over merge groups of V_G * rho'_G, level 0/1. */
double oc_mass(const oc_model *m, int level) {
  double s = 0.0;
  for (long c = 0; c < m->ncell; c++)
    if (m->cls[c] != C_UG && m->root[c] == c) s += m->vg[c] * m->rp[level][c];
  return s;
}

int oc_nsteps(const oc_model *m) { return m->nsteps; }
