// Internal definitions shared by the CUDA translation units of libcutcell.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/cutcell.h"

namespace cc {

constexpr int GH = 4;          // ghost width of every padded array (y and z; at least this in x)
// x offset of cell 0 in a padded row: with it, and rows of a multiple of 4
// values, the halo row of a tile (cells i0-2 .. for i0 a multiple of 4) starts
// on a 16-byte boundary
constexpr int GX = 6;
constexpr int HOST_GZ = 2;     // corner levels below floor / above lid in host arrays
constexpr int NFIELD = 5;      // rho', p', rho u, rho v, rho w
constexpr int NBUF = 4;        // rotating time levels
constexpr int TILE_X = 32;                          // full-cell stencil tile width (x)
// full-cell stencil schedules: tile height (y) and the number of work items
// to aim for per launch (the z-chunk length follows); the autotuner times them
// on the model's own state and keeps the fastest per launch group
constexpr int NSCHED = 4;
constexpr int SCHED_TY_F32[NSCHED] = {16, 8, 16, 8};
constexpr int SCHED_TY_F64[NSCHED] = {8, 4, 8, 4};
constexpr int SCHED_ITEMS[NSCHED] = {2 * 152, 2 * 152, 6 * 152, 6 * 152};

// cell classes and corner classes
enum : int8_t { C_UG = 0, C_FULL = 1, C_CUT = 2, C_ABS = 3 };
enum : int8_t { V_UG = 0, V_PRED = 1, V_MF = 2, V_LID = 3 };
constexpr int KB_NONE = -1000;

// Reach of the artificial-diffusion stencils in one padded column (Sec 2.1:
// fourth order; Sec 2.4: second order where a cell lacks the neighbouring
// fluid points the fourth-order term needs).  Fluid points: cells owning their
// pressure point (full or cut) and corners above the terrain, below the lid.
// In a column the cell classes run below-terrain, absorbed, cut, full from the
// floor up, so a cell is a fluid point from the column's lowest full or cut
// level on, and a corner from the lowest level above the terrain.
struct DiffCol {
  int16_t lo, hi;        // levels lo <= k < hi: the cell and the corner of this column take the
                         // fourth-order term on every axis
  int16_t ctop, vtop;    // cells k >= ctop and corners K >= vtop are not fluid points (the lid)
  int16_t c0, v0;        // this column: lowest fluid cell level, lowest fluid corner level
  int16_t cx[4], cy[4];  // lowest fluid cell level of the columns at offsets -2, -1, +1, +2 in x, in y
  int16_t vx[4], vy[4];  // lowest fluid corner level of the same columns
};

// Device-side description of one domain.  Pointers are device pointers;
// field arrays are of the model's precision (double or float).
struct DomDev {
  int nx, ny, nz;
  int px, py, pz;            // padded extents: px = nx + GX + 4 rounded up to a multiple of 8 (32-byte FP32 rows), py = ny + 2*GH, pz = nz + 2*GH
  long long plane;           // px*py
  long long ncellp;          // px*py*pz
  double dx, dy, dz, dt;
  double U, g, p0, R, cp;
  double kap;                // R/cp
  double cvcp;               // cv/cp
  double Cp;                 // cp R / cv
  double kdif;               // c4 / (16 dt)
  double ra_nu;              // Robert-Asselin coefficient
  int bc_slip;
  int periodic;              // lateral indices wrap (cyclic boundaries)
  int gox, goy;              // origin of this block in its level's box (cells; 0 for a whole level):
                             // the geometry forms positions from the level's indices
  int lid;                   // the top is the rigid lid (else a refinement face)
  // computed region: cells ci0 <= i < ci1, cj0 <= j < cj1, 0 <= k < ck1;
  // corner columns qi0 <= I < ci1, qj0 <= J < cj1
  int ci0, ci1, cj0, cj1, ck1, qi0, qj0;
  double ztop;               // height of the domain top (sponge)
  void *f[NBUF][NFIELD];     // prognostic fields, padded layout
  void *ub[NBUF];            // boundary-point velocity per level, 3 per padded column
  // base state per padded level, precision of the model
  const void *rhob, *pb, *thb, *pik, *rhobc, *tau, *ipb;
  // binomial-series coefficients C(a, 1..7) and the exponent a, for
  // (1 + x)^a - 1 with a = cv/cp (rho theta) and a = R/cp (Exner factor)
  float sth[8], sex[8];
  // the same series in FP64: C(a, 1..12) and the exponent a
  double dsth[13], dsex[13];
  // geometry (FP64 / int), padded cell layout unless noted
  const double *h;           // corner heights, ny*nx (periodic)
  const double *vf;          // nz*ny*nx interior layout (cell id)
  const double *ax, *ay;     // nz*ny*nx
  const double *az;          // (nz+1)*ny*nx
  const int8_t *cls;         // nz*ny*nx
  const int32_t *root;       // nz*ny*nx, cell id of host or -1
  const int32_t *kug;        // padded columns: cells k < kug are below the terrain
  const int8_t *vcls;        // corner classes, padded layout
  const int32_t *bK, *bI, *bJ;  // padded columns
  const double *ba, *bb, *bn;   // padded columns (bn: 3 per column)
  const int32_t *mK;         // padded corner layout
  const double *mg;          // padded corner layout
  const int32_t *ktop;       // padded columns: highest non-predicted corner level below the top
  // padded columns: corners K <= kb lie at or below the terrain and move with
  // the boundary-point velocity u_B of their column; KB_NONE where the column's
  // corners are not integrated (frame of a refined box)
  const int32_t *kb;
  const DiffCol *dcol;       // padded columns: reach of the diffusion stencils
};

// (block, tile) work item of the full-cell stencil
struct WorkItem {
  int dom, i0, j0, k0, k1, pad0, pad1, pad2;
};

// column work item of the velocity diagnosis
struct ColItem {
  int dom, I, J, pad;
};

// merge group record
struct GroupRec {
  int dom;
  int host;      // cell id (interior layout) of the host
  int start;     // index into the member array
  int count;
  double vg;     // group volume
};

__host__ __device__ inline long long pidx(const DomDev &D, int i, int j, int k) {
  return ((long long)(k + GH) * D.py + (j + GH)) * D.px + (i + GX);
}
__host__ __device__ inline int wrapi(int i, int n) {
  int r = i % n;
  return r < 0 ? r + n : r;
}
__host__ __device__ inline long long cid(const DomDev &D, int i, int j, int k) {
  return ((long long)k * D.ny + j) * D.nx + i;
}
// padded column index
__host__ __device__ inline long long qidx(const DomDev &D, int I, int J) {
  return (long long)(J + GH) * D.px + (I + GX);
}

// ---- deterministic compensated reductions (diagnostics, noalloc.cu)
#ifdef __CUDACC__
// Neumaier's running compensated sum of one thread's elements.
template <typename T>
struct NSum {
  T s, c;
  __device__ void add(T x) {
    T t = s + x;
    if (fabs((double)s) >= fabs((double)x)) c += (s - t) + x;
    else c += (x - t) + s;
    s = t;
  }
};
// A compensated partial sum s + c.  Two partials combine by TwoSum (Knuth):
// the rounding error of s1 + s2 is exact and symmetric in the operands, so a
// xor-butterfly over a warp leaves the same bits in every lane, and the
// whole reduction is the same on every run.
struct CSum {
  double s, c;
};
__device__ __forceinline__ CSum csum_add(CSum a, CSum b) {
  const double t = a.s + b.s;
  const double bp = t - a.s;
  const double e = (a.s - (t - bp)) + (b.s - bp);
  return CSum{t, (a.c + b.c) + e};
}
__device__ __forceinline__ CSum warp_csum(CSum v) {
#pragma unroll
  for (int m = 16; m >= 1; m >>= 1)
    v = csum_add(v, CSum{__shfl_xor_sync(0xffffffffu, v.s, m), __shfl_xor_sync(0xffffffffu, v.c, m)});
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int m = 16; m >= 1; m >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, m));
  return v;
}
// Block of NT threads (a multiple of 32, at most 1024): the warps' sums, then
// warp 0 over them; the result is valid in warp 0.  sh holds NT/32 entries.
template <int NT>
__device__ __forceinline__ CSum block_csum(CSum v, CSum *sh) {
  v = warp_csum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sh[w] = v;
  __syncthreads();
  if (w == 0) v = warp_csum(l < NT / 32 ? sh[l] : CSum{0.0, 0.0});
  __syncthreads();
  return v;
}
template <int NT>
__device__ __forceinline__ double block_max(double v, double *sh) {
  v = warp_max(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sh[w] = v;
  __syncthreads();
  if (w == 0) v = warp_max(l < NT / 32 ? sh[l] : 0.0);
  __syncthreads();
  return v;
}
#endif

// ---- refinement (step.cu)
// A coarse face on the boundary of a refined box: the coarse cell on the
// active side, the face (axis, side) seen from that cell, and the first of
// the 2x2 fine faces that cover it (padded coordinates of the fine cell on
// the high side of the fine face).
struct IfaceFace {
  int ax;          // 0, 1, 2
  int fi, fj, fk;  // fine face: the x-face of fine cell (fi, fj, fk) etc.
};
// coarse cell on either side of a box boundary, with up to three interface faces
struct IfaceCell {
  int i, j, k;     // coarse cell
  int slot[6];     // register slot of face (ax*2 + side), -1 if not an interface face
};
struct LevelLink {
  const DomDev *dc, *df;     // device pointers of the coarse and fine level
  int ox, oy;                // fine cell i covers coarse cell (i + ox) / 2
  const long long *pcell;    // fine padded offsets of prolonged ghost cells
  long long npcell;
  const long long *pcorn;    // fine padded offsets of prolonged ghost corners
  long long npcorn;
  const long long *rcell;    // coarse padded offsets of restricted cells
  long long nrcell;
  const long long *rcorn;    // coarse padded offsets of restricted corners
  long long nrcorn;
  const IfaceFace *faces;    // interface faces (register slots)
  int nfaces;
  const IfaceCell *icells;
  int nicells;
  void *regm, *regh;         // register sums per face (model precision)
};
// Same-level copy between sibling blocks of a level (Sec 2.2): a point of a
// block's ghost shell that lies in a sibling takes the sibling's value.
// kind: XCH_CELL (rho', p' at a cell), XCH_CORNER (the three momenta at a
// corner), XCH_COLUMN (the boundary-point velocity of a corner column; the
// offsets are padded column indices).  Offsets are padded indices of the
// destination and the source domain.
enum { XCH_CELL = 0, XCH_CORNER = 1, XCH_COLUMN = 2 };
struct XchItem {
  int32_t dst, src;
  uint16_t ddom, sdom;
  int32_t kind;
};
// copies the listed points of the two time levels r0 and r1 (ub: r1 only)
cudaError_t launch_exchange(const DomDev *d_doms, const XchItem *items, long long n, int prec, int r0, int r1,
                            cudaStream_t st);
// the links of one level's domains (a box, or its blocks) in device memory,
// with the longest list of each kind; the operations below run all of them
// in one launch
struct LinkSet {
  const LevelLink *links;
  int n;
  long long maxp, maxr, maxf, maxi;  // prolonged points, restricted points, faces, interface cells
};
cudaError_t launch_prolong(const LinkSet &S, int prec, int rC, cudaStream_t st);
cudaError_t launch_restrict(const LinkSet &S, int prec, int rF, cudaStream_t st);
cudaError_t launch_register_add(const LinkSet &S, int prec, int rF, cudaStream_t st);
cudaError_t launch_register_clear(const LinkSet &S, int prec, cudaStream_t st);
cudaError_t launch_iface(const LinkSet &S, int prec, int rO, int rC, int rN, int rF, int first,
                         cudaStream_t st);
cudaError_t launch_mass_active(const DomDev &D, const DomDev *d_dom, int prec, int rC, int rO, int both,
                               int bx0, int bx1, int by0, int by1, int bz1, double *d_out, cudaStream_t st);
cudaError_t launch_flat_columns(const DomDev &D, cudaStream_t st);
// per-column reach of the diffusion stencils (after the classes and kb exist)
cudaError_t launch_diffcols(const DomDev &D, cudaStream_t st);

// geometry of one domain (geometry.cu); returns the group list of the domain
// as device allocations owned by the caller
cudaError_t geom_build_one(DomDev &D, cudaStream_t st, int dom, int *d_err, int32_t **members_out,
                           GroupRec **recs_out, int *ng_out, int *nm_out);

// Equation-of-state coefficients shared by every domain of a model (R, cp
// and p0 are the same for all), passed to the step kernels as parameters
struct Eos {
  float sth[8], sex[8];  // binomial coefficients of (1+x)^(cv/cp) - 1 and (1+x)^(R/cp) - 1, then the exponent
  double dsth[13], dsex[13];  // the same in FP64, 12 terms
  double p0, p0R, cvcp, kap;
};

// step kernels (step.cu)
struct StepLaunch {
  const DomDev *d_doms;
  const WorkItem *items;   // the full-cell work items (FP32: those of refined boxes, staged by TMA)
  int nitems;
  const WorkItem *witems;  // FP32: the items of periodic domains (cyclic gather)
  int nwitems;
  const GroupRec *groups;
  int ngroups;
  const int32_t *members;
  const ColItem *cols;
  int ncols;
  int ndom;
  Eos eos;
  int ty;                  // tile height of the work items
  int roles;               // FP32: warp roles per block of the full-cell stencil (1, or 2: scalars and momenta apart)
  unsigned *watch;         // step watchdog flags (CC_WATCH_*), or null
  const unsigned char *tmaps;  // FP32: two 128-byte TMA tensor maps per domain (tile heights 8, 16)
  unsigned stall_tx;           // extra bytes every TMA plane barrier expects (0; the watchdog's test only)
};
// step watchdog flags, set by the full-cell stencil
constexpr unsigned WATCH_NONFINITE = 1u;  // a non-finite value was written
constexpr unsigned WATCH_COURANT = 2u;    // advective Courant number sum_d |u_d| dt / d_d above 1
constexpr unsigned WATCH_TIMEOUT = 4u;    // a bounded wait inside a kernel ran out (the step is void)
cudaError_t launch_base(const DomDev &D, int prec, double theta0, double N, double p_surf,
                        double sponge_frac, double tau_max, cudaStream_t st);
cudaError_t launch_full(const StepLaunch &L, int prec, int rO, int rC, int rN, int rF, int first,
                        cudaStream_t st);
cudaError_t launch_groups(const StepLaunch &L, int prec, int rO, int rC, int rN, int rF, int first,
                          cudaStream_t st);
cudaError_t launch_diagnose(const StepLaunch &L, int prec, int rV, int rC, int rO, int rF, int first,
                            int filter, cudaStream_t st);
int sched_tile_y(int prec, int s);
// shared-memory limits of every full-cell kernel variant (before any capture)
cudaError_t full_prepare(int prec);
cudaError_t launch_init_momentum(const DomDev &D, const DomDev *d_dom, int prec, int r, double U,
                                 cudaStream_t st);
// derived output: corner velocity component which = 0..2 (K = 0 .. nz) or the
// cell potential-temperature perturbation (which = 3), FP64 host layout
cudaError_t launch_derived(const DomDev &D, const DomDev *d_dom, int prec, int r, int which, double *d_out,
                           cudaStream_t st);
// heat content: d_out[0] sum, d_out[1] compensation; d_part 2 * 256 doubles
cudaError_t launch_heat(const DomDev *d_dom, int prec, int r, double *d_out, double *d_part, cudaStream_t st);
// error norms: d_out[0] = sum |d|, d_out[1] = sum d^2 over the corners of a
// shared with b (spacing ratio p/q: corner q I' of a is corner p I' of b) with
// K >= kmin; d_part 4 * 256 doubles
cudaError_t launch_norms(const DomDev *a, int prec_a, int ra, const DomDev *b, int prec_b, int rb, int which, int p,
                         int q, int kmin, double *d_out, double *d_part, cudaStream_t st);
// analytic hill at the corners (I dx - xc, J dy - yc), ny*nx doubles
cudaError_t launch_hill(double *h, int nx, int ny, double dx, double dy, int kind, double h0, double a, double xc,
                        double yc, cudaStream_t st);
cudaError_t launch_diag_reduce(const DomDev &D, const DomDev *d_dom, int prec, int r, double *d_out,
                               cudaStream_t st);

}  // namespace cc
