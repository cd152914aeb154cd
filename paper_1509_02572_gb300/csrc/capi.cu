// C ABI of the cut-cell library: model creation, device memory, geometry,
// state transfer, time stepping and diagnostics (declarations and the paper
// references are in include/cutcell.h).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "cc_internal.h"

using namespace cc;

namespace {

struct DomHost {
  cc_config cfg{};
  DomDev D{};
  std::vector<void *> allocs;
  bool terrain = false;
  int ng = 0, nm = 0;
  std::vector<int32_t> ghost, gstart, gmem;
};

thread_local std::string g_create_error;

}  // namespace

struct cc_model {
  int ndom = 0;
  int prec = CC_FP64;
  size_t esz = 8;
  cudaStream_t st = nullptr;
  std::vector<DomHost> dom;
  DomDev *d_doms = nullptr;
  WorkItem *d_items = nullptr;
  int nitems = 0;
  GroupRec *d_groups = nullptr;
  int ngroups = 0;
  int32_t *d_members = nullptr;
  ColItem *d_cols = nullptr;
  int ncols = 0;
  long long ghost_points = 0;
  int r[4] = {0, 1, 2, 3};  // roles: old (filtered n-1), current, new, filtered n
  long long nsteps = 0;
  long long last_launches = 0;
  bool geom = false, state = false;
  // kernel timing with CUDA events on the model's stream (cc_profile_*)
  bool prof = false;
  std::vector<cudaEvent_t> ev_pool;
  struct Ev { int kid; cudaEvent_t a, b; };
  std::vector<Ev> ev_used;
  double *d_diag = nullptr;     // 8 results + partials
  double *d_stage = nullptr;    // FP64 staging for host transfers
  size_t stage_elems = 0;
  int *d_err = nullptr;
  std::string err;
  std::vector<void *> allocs;
};

namespace {

cc_status fail(cc_model *m, cc_status s, const std::string &msg) {
  if (m) m->err = msg;
  else g_create_error = msg;
  return s;
}

cc_status cuda_fail(cc_model *m, cudaError_t e, const char *where) {
  std::string msg = std::string(where) + ": " + cudaGetErrorString(e);
  return fail(m, e == cudaErrorMemoryAllocation ? CC_ENOMEM : CC_ECUDA, msg);
}

#define CK(m, call, where)                          \
  do {                                              \
    cudaError_t e_ = (call);                        \
    if (e_ != cudaSuccess) return cuda_fail(m, e_, where); \
  } while (0)

template <typename P>
cudaError_t dalloc(std::vector<void *> &list, P **p, size_t bytes, cudaStream_t st) {
  void *q = nullptr;
  cudaError_t e = cudaMalloc(&q, bytes > 0 ? bytes : 16);
  if (e != cudaSuccess) return e;
  list.push_back(q);
  e = cudaMemsetAsync(q, 0, bytes > 0 ? bytes : 16, st);
  *p = (P *)q;
  return e;
}

bool valid_cfg(const cc_config &c, std::string &why) {
  if (c.nx < 4 || c.ny < 4 || c.nz < 4) { why = "nx, ny, nz must be >= 4"; return false; }
  if ((long long)c.nx * c.ny * c.nz > (1LL << 31) - 1) { why = "domain too large for 32-bit cell ids"; return false; }
  if (!(c.dx > 0 && c.dy > 0 && c.dz > 0 && c.dt > 0)) { why = "dx, dy, dz, dt must be > 0"; return false; }
  if (!(c.p0 > 0 && c.R > 0 && c.cp > c.R && c.g >= 0 && c.theta0 > 0 && c.p_surf > 0)) {
    why = "invalid thermodynamic constants"; return false;
  }
  if (c.N < 0 || c.ra_nu < 0 || c.ra_nu >= 0.5 || c.c4 < 0 || c.sponge_frac < 0 || c.sponge_frac >= 1 ||
      c.tau_max < 0) {
    why = "invalid N, ra_nu, c4 or sponge parameters"; return false;
  }
  if (c.N > 0 && c.g <= 0) { why = "N > 0 needs g > 0"; return false; }
  return true;
}

// ---------------------------------------------------------------- transfer kernels
// host layout (interior, corner levels from -HOST_GZ) <-> padded layout
template <typename T>
__global__ void k_scatter(const double *src, T *dst, DomDev D, int nlev, int k_first) {
  long long n = (long long)D.nx * D.ny * nlev;
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  int i = (int)(t % D.nx), j = (int)((t / D.nx) % D.ny), k = (int)(t / ((long long)D.nx * D.ny)) + k_first;
  dst[pidx(D, i, j, k)] = (T)src[t];
}
template <typename T>
__global__ void k_gather(const T *src, double *dst, DomDev D, int nlev, int k_first) {
  long long n = (long long)D.nx * D.ny * nlev;
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  int i = (int)(t % D.nx), j = (int)((t / D.nx) % D.ny), k = (int)(t / ((long long)D.nx * D.ny)) + k_first;
  dst[t] = (double)src[pidx(D, i, j, k)];
}
template <typename T>
__global__ void k_cvt_to(const double *src, T *dst, long long n) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) dst[t] = (T)src[t];
}
template <typename T>
__global__ void k_cvt_from(const T *src, double *dst, long long n) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) dst[t] = (double)src[t];
}
template <typename P>
__global__ void k_gather_raw(const P *src, P *dst, DomDev D, int nlev, int k_first) {
  long long n = (long long)D.nx * D.ny * nlev;
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  int i = (int)(t % D.nx), j = (int)((t / D.nx) % D.ny), k = (int)(t / ((long long)D.nx * D.ny)) + k_first;
  dst[t] = src[pidx(D, i, j, k)];
}

inline unsigned nb256(long long n) { return (unsigned)((n + 255) / 256); }

StepLaunch make_launch(const cc_model *m) {
  StepLaunch L{};
  L.d_doms = m->d_doms;
  L.items = m->d_items;
  L.nitems = m->nitems;
  L.groups = m->d_groups;
  L.ngroups = m->ngroups;
  L.members = m->d_members;
  L.cols = m->d_cols;
  L.ncols = m->ncols;
  L.ndom = m->ndom;
  L.ghost_points = m->ghost_points;
  L.ghost_off = nullptr;
  return L;
}

}  // namespace

extern "C" {

cc_status cc_create(const cc_config *cfgs, int n, int precision, void *stream, cc_model **out) {
  if (!out) return fail(nullptr, CC_EINVAL, "out is NULL");
  *out = nullptr;
  if (!cfgs || n <= 0) return fail(nullptr, CC_EINVAL, "need at least one domain");
  if (precision != CC_FP64 && precision != CC_FP32) return fail(nullptr, CC_EINVAL, "precision must be CC_FP64 or CC_FP32");
  for (int d = 0; d < n; d++) {
    std::string why;
    if (!valid_cfg(cfgs[d], why)) return fail(nullptr, CC_EINVAL, "domain " + std::to_string(d) + ": " + why);
  }
  cc_model *m = new cc_model();
  m->ndom = n;
  m->prec = precision;
  m->esz = precision == CC_FP64 ? 8 : 4;
  m->st = (cudaStream_t)stream;
  m->dom.resize(n);
  cudaError_t e = cudaSuccess;
  auto bail = [&](cudaError_t ee, const char *where) {
    std::string msg = std::string(where) + ": " + cudaGetErrorString(ee);
    cc_destroy(m);
    return fail(nullptr, ee == cudaErrorMemoryAllocation ? CC_ENOMEM : CC_ECUDA, msg);
  };
  size_t max_stage = 16;
  for (int d = 0; d < n; d++) {
    DomHost &H = m->dom[d];
    H.cfg = cfgs[d];
    const cc_config &c = H.cfg;
    DomDev &D = H.D;
    D.nx = c.nx; D.ny = c.ny; D.nz = c.nz;
    D.px = c.nx + 2 * GH; D.py = c.ny + 2 * GH; D.pz = c.nz + 2 * GH;
    D.plane = (long long)D.px * D.py;
    D.ncellp = D.plane * D.pz;
    D.dx = c.dx; D.dy = c.dy; D.dz = c.dz; D.dt = c.dt;
    D.U = c.U; D.g = c.g; D.p0 = c.p0; D.R = c.R; D.cp = c.cp;
    D.kap = c.R / c.cp;
    D.cvcp = (c.cp - c.R) / c.cp;
    D.Cp = c.cp * c.R / (c.cp - c.R);
    D.kdif = c.c4 / (16.0 * c.dt);
    D.ra_nu = c.ra_nu;
    D.bc_slip = c.bc_slip;
    long long ncol = (long long)c.nx * c.ny, ncell = ncol * c.nz;
    for (int b = 0; b < NBUF; b++) {
      for (int f = 0; f < NFIELD; f++)
        if ((e = dalloc(H.allocs, &D.f[b][f], D.ncellp * m->esz, m->st)) != cudaSuccess) return bail(e, "field alloc");
      if ((e = dalloc(H.allocs, &D.ub[b], 3 * ncol * m->esz, m->st)) != cudaSuccess) return bail(e, "ub alloc");
    }
    void *bt[7];
    for (int a = 0; a < 7; a++)
      if ((e = dalloc(H.allocs, &bt[a], (size_t)D.pz * m->esz, m->st)) != cudaSuccess) return bail(e, "base alloc");
    D.rhob = bt[0]; D.pb = bt[1]; D.thb = bt[2]; D.pik = bt[3]; D.rhobc = bt[4]; D.tau = bt[5]; D.ipb = bt[6];
    // binomial coefficients C(a, n), n = 1..7, of (1 + x)^a - 1
    for (int w = 0; w < 2; w++) {
      double a = w == 0 ? D.cvcp : D.kap, cn = 1.0;
      float *out = w == 0 ? D.sth : D.sex;
      for (int nn = 1; nn <= 7; nn++) {
        cn = cn * (a - (nn - 1)) / nn;
        out[nn - 1] = (float)cn;
      }
      out[7] = (float)a;
    }
    double *h, *vf, *ax, *ay, *az, *ba, *bb, *bn, *mg;
    int8_t *cls, *vcls;
    int32_t *root, *kug, *bK, *bI, *bJ, *mK, *ktop;
    if ((e = dalloc(H.allocs, &h, ncol * 8, m->st)) ||
        (e = dalloc(H.allocs, &vf, ncell * 8, m->st)) || (e = dalloc(H.allocs, &ax, ncell * 8, m->st)) ||
        (e = dalloc(H.allocs, &ay, ncell * 8, m->st)) ||
        (e = dalloc(H.allocs, &az, ncol * (c.nz + 1) * 8, m->st)) ||
        (e = dalloc(H.allocs, &cls, ncell, m->st)) || (e = dalloc(H.allocs, &root, ncell * 4, m->st)) ||
        (e = dalloc(H.allocs, &kug, ncol * 4, m->st)) || (e = dalloc(H.allocs, &vcls, D.ncellp, m->st)) ||
        (e = dalloc(H.allocs, &bK, ncol * 4, m->st)) || (e = dalloc(H.allocs, &bI, ncol * 4, m->st)) ||
        (e = dalloc(H.allocs, &bJ, ncol * 4, m->st)) || (e = dalloc(H.allocs, &ba, ncol * 8, m->st)) ||
        (e = dalloc(H.allocs, &bb, ncol * 8, m->st)) || (e = dalloc(H.allocs, &bn, 3 * ncol * 8, m->st)) ||
        (e = dalloc(H.allocs, &mK, D.ncellp * 4, m->st)) || (e = dalloc(H.allocs, &mg, D.ncellp * 8, m->st)) ||
        (e = dalloc(H.allocs, &ktop, ncol * 4, m->st)))
      return bail(e, "geometry alloc");
    D.h = h; D.vf = vf; D.ax = ax; D.ay = ay; D.az = az; D.cls = cls; D.root = root; D.kug = kug;
    D.vcls = vcls; D.bK = bK; D.bI = bI; D.bJ = bJ; D.ba = ba; D.bb = bb; D.bn = bn; D.mK = mK; D.mg = mg;
    D.ktop = ktop;
    if ((e = launch_base(D, precision, c.theta0, c.N, c.p_surf, c.sponge_frac, c.tau_max, m->st)) != cudaSuccess)
      return bail(e, "base state");
    max_stage = std::max(max_stage, (size_t)(ncol * (c.nz + 1 + 2 * HOST_GZ)));
    max_stage = std::max(max_stage, (size_t)(ncol * (c.nz + 1)));
    long long frame = D.plane - ncol;
    m->ghost_points = std::max(m->ghost_points, frame * D.pz);
  }
  // device domain table
  if ((e = dalloc(m->allocs, &m->d_doms, sizeof(DomDev) * n, m->st)) != cudaSuccess) return bail(e, "domain table");
  {
    std::vector<DomDev> hd(n);
    for (int d = 0; d < n; d++) hd[d] = m->dom[d].D;
    if ((e = cudaMemcpyAsync(m->d_doms, hd.data(), sizeof(DomDev) * n, cudaMemcpyHostToDevice, m->st)) != cudaSuccess)
      return bail(e, "domain table copy");
    if ((e = cudaStreamSynchronize(m->st)) != cudaSuccess) return bail(e, "sync");
  }
  // (domain, tile, z-chunk) work list of the full-cell stencil: z is split so
  // that every SM gets several work items
  {
    const int TILE_Y = full_tile_y(precision);
    long long tiles = 0;
    for (auto &H : m->dom)
      tiles += (long long)((H.D.nx + TILE_X - 1) / TILE_X) * ((H.D.ny + TILE_Y - 1) / TILE_Y);
    const long long want = 2 * 152;
    long long splits = std::max(1LL, (want + tiles - 1) / tiles);
    std::vector<WorkItem> items;
    for (int d = 0; d < n; d++) {
      const DomDev &D = m->dom[d].D;
      int chunk = (int)std::max(8LL, (D.nz + splits - 1) / splits);
      for (int k0 = 0; k0 < D.nz; k0 += chunk)
        for (int j0 = 0; j0 < D.ny; j0 += TILE_Y)
          for (int i0 = 0; i0 < D.nx; i0 += TILE_X) {
            WorkItem w{};
            w.dom = d; w.i0 = i0; w.j0 = j0; w.k0 = k0; w.k1 = std::min(D.nz, k0 + chunk);
            items.push_back(w);
          }
    }
    m->nitems = (int)items.size();
    if ((e = dalloc(m->allocs, &m->d_items, sizeof(WorkItem) * items.size(), m->st)) != cudaSuccess)
      return bail(e, "work list");
    if ((e = cudaMemcpyAsync(m->d_items, items.data(), sizeof(WorkItem) * items.size(), cudaMemcpyHostToDevice,
                             m->st)) != cudaSuccess)
      return bail(e, "work list copy");
    std::vector<ColItem> cols;
    for (int d = 0; d < n; d++)
      for (int J = 0; J < m->dom[d].D.ny; J++)
        for (int I = 0; I < m->dom[d].D.nx; I++) cols.push_back(ColItem{d, I, J, 0});
    m->ncols = (int)cols.size();
    if ((e = dalloc(m->allocs, &m->d_cols, sizeof(ColItem) * cols.size(), m->st)) != cudaSuccess)
      return bail(e, "column list");
    if ((e = cudaMemcpyAsync(m->d_cols, cols.data(), sizeof(ColItem) * cols.size(), cudaMemcpyHostToDevice,
                             m->st)) != cudaSuccess)
      return bail(e, "column list copy");
    if ((e = cudaStreamSynchronize(m->st)) != cudaSuccess) return bail(e, "sync");
  }
  if ((e = dalloc(m->allocs, &m->d_diag, sizeof(double) * (8 + 5 * 256), m->st)) != cudaSuccess) return bail(e, "diag");
  if ((e = dalloc(m->allocs, &m->d_stage, sizeof(double) * max_stage, m->st)) != cudaSuccess) return bail(e, "stage");
  m->stage_elems = max_stage;
  if ((e = dalloc(m->allocs, &m->d_err, sizeof(int), m->st)) != cudaSuccess) return bail(e, "err flag");
  if ((e = cudaStreamSynchronize(m->st)) != cudaSuccess) return bail(e, "sync");
  *out = m;
  return CC_OK;
}

cc_status cc_destroy(cc_model *m) {
  if (!m) return CC_OK;
  if (m->st || true) cudaStreamSynchronize(m->st);
  for (auto &H : m->dom)
    for (void *p : H.allocs) cudaFree(p);
  for (void *p : m->allocs) cudaFree(p);
  cudaFree(m->d_groups);
  cudaFree(m->d_members);
  for (auto &e : m->ev_used) {
    cudaEventDestroy(e.a);
    cudaEventDestroy(e.b);
  }
  for (auto e : m->ev_pool) cudaEventDestroy(e);
  delete m;
  return CC_OK;
}

const char *cc_last_error(const cc_model *m) {
  if (!m) return g_create_error.c_str();
  return m->err.c_str();
}

cc_status cc_set_terrain(cc_model *m, int d, const double *corner_h) {
  if (!m || !corner_h) return fail(m, CC_EINVAL, "null argument");
  if (d < 0 || d >= m->ndom) return fail(m, CC_EINVAL, "domain index out of range");
  DomHost &H = m->dom[d];
  long long ncol = (long long)H.cfg.nx * H.cfg.ny;
  double top = H.cfg.nz * H.cfg.dz;
  for (long long q = 0; q < ncol; q++) {
    double v = corner_h[q];
    if (!std::isfinite(v) || v < 0.0 || v >= top)
      return fail(m, CC_EINVAL, "terrain heights must be finite, >= 0 and below the lid");
  }
  CK(m, cudaMemcpyAsync((void *)H.D.h, corner_h, ncol * 8, cudaMemcpyHostToDevice, m->st), "terrain copy");
  CK(m, cudaStreamSynchronize(m->st), "terrain sync");
  H.terrain = true;
  m->geom = false;
  m->state = false;
  return CC_OK;
}

cc_status cc_build_geometry(cc_model *m) {
  if (!m) return fail(m, CC_EINVAL, "null model");
  for (auto &H : m->dom)
    if (!H.terrain) return fail(m, CC_ESTATE, "terrain not set for every domain");
  cudaFree(m->d_groups);
  cudaFree(m->d_members);
  m->d_groups = nullptr;
  m->d_members = nullptr;
  std::vector<GroupRec> all;
  std::vector<int32_t> allm;
  for (int d = 0; d < m->ndom; d++) {
    DomHost &H = m->dom[d];
    CK(m, cudaMemsetAsync(m->d_err, 0, sizeof(int), m->st), "err reset");
    int32_t *mem = nullptr;
    GroupRec *recs = nullptr;
    int ng = 0, nm = 0;
    cudaError_t e = geom_build_one(H.D, m->st, d, m->d_err, &mem, &recs, &ng, &nm);
    if (e != cudaSuccess) return cuda_fail(m, e, "geometry");
    int herr = 0;
    CK(m, cudaMemcpy(&herr, m->d_err, sizeof(int), cudaMemcpyDeviceToHost), "err read");
    std::vector<GroupRec> r(ng);
    std::vector<int32_t> mm(nm);
    if (ng) CK(m, cudaMemcpy(r.data(), recs, sizeof(GroupRec) * ng, cudaMemcpyDeviceToHost), "groups read");
    if (nm) CK(m, cudaMemcpy(mm.data(), mem, sizeof(int32_t) * nm, cudaMemcpyDeviceToHost), "members read");
    cudaFree(mem);
    cudaFree(recs);
    if (herr) {
      std::string why = "domain " + std::to_string(d) + ":";
      if (herr & 1) why += " vertical merge target above the lid;";
      if (herr & 2) why += " merge chain ends below the terrain or loops;";
      if (herr & 4) why += " terrain reaches the level below the lid;";
      if (herr & 8) why += " no nearest plane of predicted points for a boundary point;";
      if (herr & 16) why += " no predicted point above a merged-face point;";
      return fail(m, CC_EGEOM, why);
    }
    H.ng = ng;
    H.nm = nm;
    H.ghost.resize(ng);
    H.gstart.resize(ng + 1);
    H.gmem = mm;
    int off = (int)allm.size();
    for (int g = 0; g < ng; g++) {
      H.ghost[g] = r[g].host;
      H.gstart[g] = r[g].start;
      GroupRec q = r[g];
      q.start += off;
      all.push_back(q);
    }
    H.gstart[ng] = nm;
    allm.insert(allm.end(), mm.begin(), mm.end());
  }
  m->ngroups = (int)all.size();
  CK(m, cudaMalloc(&m->d_groups, sizeof(GroupRec) * std::max<size_t>(1, all.size())), "groups alloc");
  CK(m, cudaMalloc(&m->d_members, sizeof(int32_t) * std::max<size_t>(1, allm.size())), "members alloc");
  if (!all.empty())
    CK(m, cudaMemcpy(m->d_groups, all.data(), sizeof(GroupRec) * all.size(), cudaMemcpyHostToDevice), "groups copy");
  if (!allm.empty())
    CK(m, cudaMemcpy(m->d_members, allm.data(), sizeof(int32_t) * allm.size(), cudaMemcpyHostToDevice),
       "members copy");
  m->geom = true;
  m->state = false;
  return CC_OK;
}

cc_status cc_get_geometry(const cc_model *mc, int d, double *vf, double *ax, double *ay, double *az, int8_t *cls,
                          int32_t *root, int8_t *vcls) {
  cc_model *m = const_cast<cc_model *>(mc);
  if (!m) return fail(m, CC_EINVAL, "null model");
  if (d < 0 || d >= m->ndom) return fail(m, CC_EINVAL, "domain index out of range");
  if (!m->geom) return fail(m, CC_ESTATE, "geometry not built");
  const DomDev &D = m->dom[d].D;
  long long ncol = (long long)D.nx * D.ny, ncell = ncol * D.nz;
  if (vf) CK(m, cudaMemcpy(vf, D.vf, ncell * 8, cudaMemcpyDeviceToHost), "vf");
  if (ax) CK(m, cudaMemcpy(ax, D.ax, ncell * 8, cudaMemcpyDeviceToHost), "ax");
  if (ay) CK(m, cudaMemcpy(ay, D.ay, ncell * 8, cudaMemcpyDeviceToHost), "ay");
  if (az) CK(m, cudaMemcpy(az, D.az, ncol * (D.nz + 1) * 8, cudaMemcpyDeviceToHost), "az");
  if (cls) CK(m, cudaMemcpy(cls, D.cls, ncell, cudaMemcpyDeviceToHost), "cls");
  if (root) CK(m, cudaMemcpy(root, D.root, ncell * 4, cudaMemcpyDeviceToHost), "root");
  if (vcls) {
    int nlev = D.nz + 1 + 2 * HOST_GZ;
    int8_t *tmp = (int8_t *)m->d_stage;
    k_gather_raw<int8_t><<<nb256(ncol * nlev), 256, 0, m->st>>>(D.vcls, tmp, D, nlev, -HOST_GZ);
    CK(m, cudaGetLastError(), "vcls gather");
    CK(m, cudaMemcpyAsync(vcls, tmp, ncol * nlev, cudaMemcpyDeviceToHost, m->st), "vcls");
    CK(m, cudaStreamSynchronize(m->st), "sync");
  }
  return CC_OK;
}

cc_status cc_get_stencils(const cc_model *mc, int d, int32_t *bK, int32_t *bI, int32_t *bJ, double *ba, double *bb,
                          double *bn, int32_t *mK, double *mg) {
  cc_model *m = const_cast<cc_model *>(mc);
  if (!m) return fail(m, CC_EINVAL, "null model");
  if (d < 0 || d >= m->ndom) return fail(m, CC_EINVAL, "domain index out of range");
  if (!m->geom) return fail(m, CC_ESTATE, "geometry not built");
  const DomDev &D = m->dom[d].D;
  long long ncol = (long long)D.nx * D.ny;
  if (bK) CK(m, cudaMemcpy(bK, D.bK, ncol * 4, cudaMemcpyDeviceToHost), "bK");
  if (bI) CK(m, cudaMemcpy(bI, D.bI, ncol * 4, cudaMemcpyDeviceToHost), "bI");
  if (bJ) CK(m, cudaMemcpy(bJ, D.bJ, ncol * 4, cudaMemcpyDeviceToHost), "bJ");
  if (ba) CK(m, cudaMemcpy(ba, D.ba, ncol * 8, cudaMemcpyDeviceToHost), "ba");
  if (bb) CK(m, cudaMemcpy(bb, D.bb, ncol * 8, cudaMemcpyDeviceToHost), "bb");
  if (bn) CK(m, cudaMemcpy(bn, D.bn, 3 * ncol * 8, cudaMemcpyDeviceToHost), "bn");
  int nlev = D.nz + 1 + 2 * HOST_GZ;
  if (mK) {
    int32_t *tmp = (int32_t *)m->d_stage;
    k_gather_raw<int32_t><<<nb256(ncol * nlev), 256, 0, m->st>>>(D.mK, tmp, D, nlev, -HOST_GZ);
    CK(m, cudaGetLastError(), "mK gather");
    CK(m, cudaMemcpyAsync(mK, tmp, ncol * nlev * 4, cudaMemcpyDeviceToHost, m->st), "mK");
    CK(m, cudaStreamSynchronize(m->st), "sync");
  }
  if (mg) {
    double *tmp = m->d_stage;
    k_gather_raw<double><<<nb256(ncol * nlev), 256, 0, m->st>>>(D.mg, tmp, D, nlev, -HOST_GZ);
    CK(m, cudaGetLastError(), "mg gather");
    CK(m, cudaMemcpyAsync(mg, tmp, ncol * nlev * 8, cudaMemcpyDeviceToHost, m->st), "mg");
    CK(m, cudaStreamSynchronize(m->st), "sync");
  }
  return CC_OK;
}

cc_status cc_get_groups(const cc_model *mc, int d, int *ngroups, int *nmembers, int32_t *host, int32_t *start,
                        int32_t *members) {
  cc_model *m = const_cast<cc_model *>(mc);
  if (!m || !ngroups || !nmembers) return fail(m, CC_EINVAL, "null argument");
  if (d < 0 || d >= m->ndom) return fail(m, CC_EINVAL, "domain index out of range");
  if (!m->geom) return fail(m, CC_ESTATE, "geometry not built");
  const DomHost &H = m->dom[d];
  *ngroups = H.ng;
  *nmembers = H.nm;
  if (host) std::memcpy(host, H.ghost.data(), sizeof(int32_t) * H.ng);
  if (start) std::memcpy(start, H.gstart.data(), sizeof(int32_t) * (H.ng + 1));
  if (members) std::memcpy(members, H.gmem.data(), sizeof(int32_t) * H.nm);
  return CC_OK;
}

cc_status cc_init_state(cc_model *m) {
  if (!m) return fail(m, CC_EINVAL, "null model");
  if (!m->geom) return fail(m, CC_ESTATE, "geometry not built");
  for (auto &H : m->dom) {
    for (int b = 0; b < NBUF; b++) {
      for (int f = 0; f < NFIELD; f++)
        CK(m, cudaMemsetAsync(H.D.f[b][f], 0, H.D.ncellp * m->esz, m->st), "state reset");
      CK(m, cudaMemsetAsync(H.D.ub[b], 0, 3 * (size_t)H.D.nx * H.D.ny * m->esz, m->st), "ub reset");
    }
  }
  m->r[0] = 0; m->r[1] = 1; m->r[2] = 2; m->r[3] = 3;
  for (int d = 0; d < m->ndom; d++)
    CK(m, launch_init_momentum(m->dom[d].D, m->d_doms + d, m->prec, m->r[1], m->dom[d].cfg.U, m->st), "init momentum");
  StepLaunch L = make_launch(m);
  CK(m, launch_diagnose(L, m->prec, m->r[1], m->r[1], m->r[1], m->r[1], 1, 0, m->st), "init diagnose");
  CK(m, cudaStreamSynchronize(m->st), "init sync");
  m->nsteps = 0;
  m->state = true;
  return CC_OK;
}

static long long field_elems(const DomDev &D, int field, int *nlev, int *kfirst) {
  long long ncol = (long long)D.nx * D.ny;
  if (field == CC_RHOP || field == CC_PP) {
    *nlev = D.nz;
    *kfirst = 0;
    return ncol * D.nz;
  }
  if (field == CC_UB) {
    *nlev = 0;
    *kfirst = 0;
    return 3 * ncol;
  }
  *nlev = D.nz + 1 + 2 * HOST_GZ;
  *kfirst = -HOST_GZ;
  return ncol * (*nlev);
}

cc_status cc_upload_state(cc_model *m, int d, int field, int level, const double *host) {
  if (!m || !host) return fail(m, CC_EINVAL, "null argument");
  if (d < 0 || d >= m->ndom) return fail(m, CC_EINVAL, "domain index out of range");
  if (field < 0 || field > CC_UB || level < 0 || level > 1) return fail(m, CC_EINVAL, "bad field or level");
  if (!m->state) return fail(m, CC_ESTATE, "state not initialised");
  const DomDev &D = m->dom[d].D;
  int buf = level == 0 ? m->r[0] : m->r[1];
  int nlev, kfirst;
  long long n = field_elems(D, field, &nlev, &kfirst);
  CK(m, cudaMemcpyAsync(m->d_stage, host, n * 8, cudaMemcpyHostToDevice, m->st), "upload");
  if (field == CC_UB) {
    if (m->prec == CC_FP64) k_cvt_to<double><<<nb256(n), 256, 0, m->st>>>(m->d_stage, (double *)D.ub[buf], n);
    else k_cvt_to<float><<<nb256(n), 256, 0, m->st>>>(m->d_stage, (float *)D.ub[buf], n);
  } else {
    void *dst = D.f[buf][field];
    if (m->prec == CC_FP64) k_scatter<double><<<nb256(n), 256, 0, m->st>>>(m->d_stage, (double *)dst, D, nlev, kfirst);
    else k_scatter<float><<<nb256(n), 256, 0, m->st>>>(m->d_stage, (float *)dst, D, nlev, kfirst);
  }
  CK(m, cudaGetLastError(), "upload scatter");
  CK(m, cudaStreamSynchronize(m->st), "upload sync");
  return CC_OK;
}

cc_status cc_download_state(const cc_model *mc, int d, int field, int level, double *host) {
  cc_model *m = const_cast<cc_model *>(mc);
  if (!m || !host) return fail(m, CC_EINVAL, "null argument");
  if (d < 0 || d >= m->ndom) return fail(m, CC_EINVAL, "domain index out of range");
  if (field < 0 || field > CC_UB || level < 0 || level > 1) return fail(m, CC_EINVAL, "bad field or level");
  if (!m->state) return fail(m, CC_ESTATE, "state not initialised");
  const DomDev &D = m->dom[d].D;
  int buf = level == 0 ? m->r[0] : m->r[1];
  int nlev, kfirst;
  long long n = field_elems(D, field, &nlev, &kfirst);
  if (field == CC_UB) {
    if (m->prec == CC_FP64) k_cvt_from<double><<<nb256(n), 256, 0, m->st>>>((const double *)D.ub[buf], m->d_stage, n);
    else k_cvt_from<float><<<nb256(n), 256, 0, m->st>>>((const float *)D.ub[buf], m->d_stage, n);
  } else {
    const void *src = D.f[buf][field];
    if (m->prec == CC_FP64)
      k_gather<double><<<nb256(n), 256, 0, m->st>>>((const double *)src, m->d_stage, D, nlev, kfirst);
    else
      k_gather<float><<<nb256(n), 256, 0, m->st>>>((const float *)src, m->d_stage, D, nlev, kfirst);
  }
  CK(m, cudaGetLastError(), "download gather");
  CK(m, cudaMemcpyAsync(host, m->d_stage, n * 8, cudaMemcpyDeviceToHost, m->st), "download");
  CK(m, cudaStreamSynchronize(m->st), "download sync");
  return CC_OK;
}

}  // extern "C"

static cudaEvent_t ev_get(cc_model *m) {
  if (!m->ev_pool.empty()) {
    cudaEvent_t e = m->ev_pool.back();
    m->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

// launch one stage, bracketed by events when profiling is on
template <typename F>
static cudaError_t timed(cc_model *m, int kid, F &&launch) {
  if (!m->prof) return launch();
  cudaEvent_t a = ev_get(m), b = ev_get(m);
  if (!a || !b) return cudaErrorMemoryAllocation;
  cudaError_t e = cudaEventRecord(a, m->st);
  if (e != cudaSuccess) return e;
  e = launch();
  if (e != cudaSuccess) return e;
  e = cudaEventRecord(b, m->st);
  m->ev_used.push_back({kid, a, b});
  return e;
}

extern "C" {

cc_status cc_step(cc_model *m, int n) {
  if (!m) return fail(m, CC_EINVAL, "null model");
  if (n < 0) return fail(m, CC_EINVAL, "negative step count");
  if (!m->state) return fail(m, CC_ESTATE, "state not initialised");
  StepLaunch L = make_launch(m);
  long long nl = 0;
  for (int s = 0; s < n; s++) {
    int first = m->nsteps == 0;
    int rO = first ? m->r[1] : m->r[0];
    const int rC = m->r[1], rN = m->r[2], rF = m->r[3], pr = m->prec;
    cudaStream_t st = m->st;
    if (L.nitems > 0) {
      CK(m, timed(m, CC_K_FULL, [&] { return launch_full(L, pr, rO, rC, rN, rF, first, st); }), "full-cell stencil");
      nl++;
    }
    if (L.ngroups > 0) {
      CK(m, timed(m, CC_K_GROUPS, [&] { return launch_groups(L, pr, rO, rC, rN, rF, first, st); }), "cut cells");
      nl++;
    }
    if (L.ncols > 0) {
      CK(m, timed(m, CC_K_DIAGNOSE, [&] { return launch_diagnose(L, pr, rN, rC, rO, rF, first, 1, st); }),
         "velocity diagnosis");
      nl++;
    }
    int o = m->r[0], c = m->r[1];
    m->r[0] = m->r[3];
    m->r[1] = m->r[2];
    m->r[2] = o;
    m->r[3] = c;
    m->nsteps++;
  }
  m->last_launches = nl;
  return CC_OK;
}

cc_status cc_diagnostics(cc_model *m, int d, cc_diag *out) {
  if (!m || !out) return fail(m, CC_EINVAL, "null argument");
  if (d < 0 || d >= m->ndom) return fail(m, CC_EINVAL, "domain index out of range");
  if (!m->state) return fail(m, CC_ESTATE, "state not initialised");
  CK(m, launch_diag_reduce(m->dom[d].D, m->d_doms + d, m->prec, m->r[1], m->d_diag, m->st), "diagnostics");
  double h[8];
  CK(m, cudaMemcpyAsync(h, m->d_diag, sizeof(double) * 5, cudaMemcpyDeviceToHost, m->st), "diag copy");
  CK(m, cudaStreamSynchronize(m->st), "diag sync");
  out->mass = h[0];
  out->mass_comp = h[1];
  out->max_u = h[2];
  out->max_w = h[3];
  out->nonfinite = (long long)h[4];
  out->steps = m->nsteps;
  if (out->nonfinite > 0) return fail(m, CC_ENUMERIC, "non-finite values in the state");
  return CC_OK;
}

cc_status cc_synchronize(cc_model *m) {
  if (!m) return fail(m, CC_EINVAL, "null model");
  CK(m, cudaStreamSynchronize(m->st), "synchronize");
  return CC_OK;
}

long long cc_last_launch_count(const cc_model *m) { return m ? m->last_launches : 0; }

cc_status cc_profile_enable(cc_model *m, int on) {
  if (!m) return fail(m, CC_EINVAL, "null model");
  m->prof = on != 0;
  return CC_OK;
}

cc_status cc_profile_read(cc_model *m, int kernel, double *total_ms, long long *launches) {
  if (!m || !total_ms || !launches) return fail(m, CC_EINVAL, "null argument");
  if (kernel < 0 || kernel > CC_K_GHOST) return fail(m, CC_EINVAL, "bad kernel id");
  CK(m, cudaStreamSynchronize(m->st), "profile sync");
  double t = 0;
  long long c = 0;
  for (auto &e : m->ev_used)
    if (e.kid == kernel) {
      float ms = 0;
      CK(m, cudaEventElapsedTime(&ms, e.a, e.b), "event time");
      t += ms;
      c++;
    }
  *total_ms = t;
  *launches = c;
  return CC_OK;
}

cc_status cc_profile_reset(cc_model *m) {
  if (!m) return fail(m, CC_EINVAL, "null model");
  CK(m, cudaStreamSynchronize(m->st), "profile sync");
  for (auto &e : m->ev_used) {
    m->ev_pool.push_back(e.a);
    m->ev_pool.push_back(e.b);
  }
  m->ev_used.clear();
  return CC_OK;
}

}  // extern "C"
