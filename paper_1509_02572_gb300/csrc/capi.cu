// C ABI of the cut-cell library: model creation, device memory, geometry,
// state transfer, time stepping and diagnostics (declarations and the paper
// references are in include/cutcell.h).
#include <cuda.h>  // CUtensorMap and its enumerations (the encoder is looked up at run time)
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <type_traits>
#include <vector>

#include "cc_internal.h"

using namespace cc;

namespace {

struct DomHost {
  cc_config cfg{};
  DomDev D{};
  std::vector<void *> allocs;
  bool terrain = false;
  std::vector<double> hh;  // host copy of the corner heights
  int ng = 0, nm = 0;
  std::vector<int32_t> ghost, gstart, gmem;
  int r[4] = {0, 1, 2, 3};  // roles: old (filtered n-1), current, new, filtered n
  long long nsteps = 0;
  // this domain's ranges of the model-wide work, group and column lists
  // (FP32: the items of a refined box, staged by TMA; witem0/nwitem those of
  // a periodic domain, gathered from the cyclic indices)
  int item0[NSCHED] = {}, nitem[NSCHED] = {}, witem0[NSCHED] = {}, nwitem[NSCHED] = {};
  int group0 = 0, ngroup = 0, col0 = 0, ncol = 0;
  int sched = 0;  // full-cell schedule of this level (refined models)
  int roles = 1;  // FP32: warp roles per block of this level's stencil (refined models)
};

// Coarse-fine link of a domain of refined level l >= 1 (a level's box or one
// of its blocks) with the domain of level l-1 (host side; the LevelLink holds
// the device lists)
struct LinkHost {
  cc_box box{};                                // this domain's box, in the coarser level's frame
  int dc = 0;                                  // the coarser level's domain
  int x0 = 0, x1 = 0, y0 = 0, y1 = 0, z1 = 0;  // covered box in coarse cells
  LevelLink L{};
};

// Domains of a refined model: the level of each domain, its box relative to
// the coarser level (level >= 1), the whole box of each level, and the origin
// of each domain's block in its level's box (sibling blocks of the finest level)
struct Layout {
  std::vector<int> level;
  std::vector<cc_box> box;
  std::vector<cc_box> lev_box;
  std::vector<std::array<int, 2>> off;
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
  WorkItem *d_items[NSCHED] = {};  // work list of every full-cell schedule
  int nitems[NSCHED] = {};         // its first part (FP32: the items of refined boxes, staged by TMA)
  int nwitems[NSCHED] = {};        // FP32: the items of periodic domains (cyclic gather), after the first part
  int sched = 0;                   // schedule of the ensemble launch
  int roles = 1;                   // FP32: warp roles per block of the ensemble launch
  bool tuned = false;
  // CUDA graphs of one step (one cycle of level 0 for a refined model), keyed
  // by the time-level roles and schedules of every domain; captured on a
  // private stream, launched on the model's stream
  struct GraphEnt {
    std::vector<int> key;
    cudaGraphExec_t exec = nullptr;
    long long launches = 0;
  };
  std::vector<GraphEnt> graphs;
  bool graphs_on = true;
  bool dry = false;  // bookkeeping only (roles, step counts): the graph does the work
  cudaStream_t cap = nullptr;
  GroupRec *d_groups = nullptr;
  int ngroups = 0;
  int32_t *d_members = nullptr;
  ColItem *d_cols = nullptr;
  int ncols = 0;
  bool refined = false;
  std::vector<LinkHost> link;  // link[d] for every domain d of level >= 1 of a refined model
  // refined models: the domains of each level (consecutive), the level and
  // block origin of each domain, each level's whole box; the same-level
  // copies of each level with sibling blocks
  int nlev = 0;
  std::vector<int> lev_first, lev_count, dom_level;
  std::vector<std::array<int, 2>> blk_off;
  std::vector<cc_box> lev_box;
  std::vector<XchItem *> d_xch;
  std::vector<long long> nxch;
  std::vector<LinkSet> lset;  // the links of each level >= 1 (one launch per operation)
  Eos eos{};                   // equation-of-state coefficients of every domain
  long long last_launches = 0;
  bool geom = false, state = false;
  // kernel timing with CUDA events on the model's stream (cc_profile_*)
  bool prof = false;
  std::vector<cudaEvent_t> ev_pool;
  struct Ev { int kid; cudaEvent_t a, b; };
  std::vector<Ev> ev_used;
  double *d_diag = nullptr;     // 8 results + partials
  double *d_stage = nullptr;    // FP64 staging for host transfers
  // state uploads and downloads alternate between d_stage and d_stage2; an
  // upload's host copy runs on the transfer stream xs, so that it overlaps
  // the conversion kernel of the previous transfer on the model's stream
  double *d_stage2 = nullptr;
  cudaStream_t xs = nullptr;
  cudaEvent_t ev_copied[2] = {}, ev_staged[2] = {};
  bool used_valid[2] = {false, false};
  int xslot = 0;
  size_t stage_elems = 0;
  // whole-state uploads (cc_upload_all_*): a staging buffer of the whole
  // state, one copy event per domain, and the event after the conversions
  void *d_bulk = nullptr;
  size_t bulk_bytes = 0;
  std::vector<cudaEvent_t> ev_bulk;
  cudaEvent_t ev_bulk_done = nullptr;
  bool bulk_used = false;
  int *d_err = nullptr;
  // step watchdog (flags of the full-cell stencil): the device word, its copy
  // in pinned host memory, made after each cc_step call, and the event that
  // marks the copy complete
  unsigned *d_watch = nullptr, *h_watch = nullptr;
  cudaEvent_t ev_watch = nullptr;
  bool watch_pending = false;
  // FP32: TMA tensor maps of the two-cell stencil, two per domain (tile
  // heights 8 and 16), in device memory
  unsigned char *d_tmaps = nullptr;
  unsigned stall_tx = 0;  // cc_inject_wait_timeout

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

// The step watchdog's verdict from the host copy of its flags (valid once
// ev_watch has completed).
cc_status watch_verdict(cc_model *m) {
  const unsigned w = *m->h_watch;
  if (w & WATCH_NONFINITE) return fail(m, CC_ENUMERIC, "step watchdog: a step wrote a non-finite value");
  if (w & WATCH_COURANT)
    return fail(m, CC_ENUMERIC, "step watchdog: an advective Courant number sum |u_d| dt / d_d exceeded 1");
  if (w & WATCH_TIMEOUT)
    return fail(m, CC_ETIMEOUT, "step watchdog: a bounded wait in the full-cell stencil ran out (the step is void)");
  return CC_OK;
}

// Clears the watchdog (new state: initialisation, checkpoint load).
cc_status watch_reset(cc_model *m) {
  CK(m, cudaMemsetAsync(m->d_watch, 0, 16, m->st), "watchdog reset");
  if (m->watch_pending) CK(m, cudaEventSynchronize(m->ev_watch), "watchdog reset");
  *m->h_watch = 0;
  m->watch_pending = false;
  return CC_OK;
}


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
// host layout (interior, corner levels from -HOST_GZ) <-> padded layout;
// T the field's element type, H the host buffer's (FP64, or FP32 for FP32
// models)
template <typename T, typename H = double>
__global__ void k_scatter(const H *src, T *dst, DomDev D, int nlev, int k_first) {
  long long n = (long long)D.nx * D.ny * nlev;
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  int i = (int)(t % D.nx), j = (int)((t / D.nx) % D.ny), k = (int)(t / ((long long)D.nx * D.ny)) + k_first;
  dst[pidx(D, i, j, k)] = (T)src[t];
}
template <typename T, typename H = double>
__global__ void k_gather(const T *src, H *dst, DomDev D, int nlev, int k_first) {
  long long n = (long long)D.nx * D.ny * nlev;
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  int i = (int)(t % D.nx), j = (int)((t / D.nx) % D.ny), k = (int)(t / ((long long)D.nx * D.ny)) + k_first;
  dst[t] = (H)src[pidx(D, i, j, k)];
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

// launch description of every domain (d < 0) or of domain d alone
// The launches of every domain (lev < 0), or of level lev of a refined model
// (all its blocks: their items, groups and columns are consecutive).
StepLaunch make_launch(const cc_model *m, int lev = -1) {
  StepLaunch L{};
  L.d_doms = m->d_doms;
  L.items = m->d_items[m->sched];
  L.nitems = m->nitems[m->sched];
  L.witems = m->d_items[m->sched] + m->nitems[m->sched];
  L.nwitems = m->nwitems[m->sched];
  L.ty = sched_tile_y(m->prec, m->sched);
  L.roles = m->roles;
  L.groups = m->d_groups;
  L.ngroups = m->ngroups;
  L.members = m->d_members;
  L.cols = m->d_cols;
  L.ncols = m->ncols;
  L.ndom = m->ndom;
  L.eos = m->eos;
  L.watch = m->d_watch;
  L.tmaps = m->d_tmaps;
  L.stall_tx = m->stall_tx;
  if (lev >= 0) {
    const int d0 = m->lev_first[lev], d1 = d0 + m->lev_count[lev];
    const DomHost &H = m->dom[d0];
    const int sc = H.sched;  // the blocks of a level share one schedule
    L.items = m->d_items[sc] + H.item0[sc];
    L.witems = m->d_items[sc] + H.witem0[sc];
    L.ty = sched_tile_y(m->prec, sc);
    L.roles = H.roles;
    L.groups = m->d_groups + H.group0;
    L.cols = m->d_cols + H.col0;
    L.nitems = L.nwitems = L.ngroups = L.ncols = 0;
    for (int q = d0; q < d1; q++) {
      L.nitems += m->dom[q].nitem[sc];
      L.nwitems += m->dom[q].nwitem[sc];
      L.ngroups += m->dom[q].ngroup;
      L.ncols += m->dom[q].ncol;
    }
  }
  return L;
}

// padded columns <-> host columns (w values per column)
template <typename P>
__global__ void k_gather_cols(const P *src, P *dst, DomDev D, int w) {
  long long n = (long long)D.nx * D.ny * w;
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  int c = (int)(t % w);
  long long q = t / w;
  int I = (int)(q % D.nx), J = (int)(q / D.nx);
  dst[t] = src[qidx(D, I, J) * w + c];
}
template <typename T, typename H = double>
__global__ void k_scatter_cols(const H *src, T *dst, DomDev D, int w) {
  long long n = (long long)D.nx * D.ny * w;
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  int c = (int)(t % w);
  long long q = t / w;
  int I = (int)(q % D.nx), J = (int)(q / D.nx);
  dst[qidx(D, I, J) * w + c] = (T)src[t];
}
template <typename T, typename H = double>
__global__ void k_gather_cols_cvt(const T *src, H *dst, DomDev D, int w) {
  long long n = (long long)D.nx * D.ny * w;
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  int c = (int)(t % w);
  long long q = t / w;
  int I = (int)(q % D.nx), J = (int)(q / D.nx);
  dst[t] = (H)src[qidx(D, I, J) * w + c];
}

// corner heights of a box level must vanish within this many corners of its
// edges: the geometry of the cells near the edges is evaluated as over a flat
// floor, which the padded frame continues
constexpr int FLAT_MARGIN = 8;

// domain kinds: a periodic block with the lid (ensemble member, level 0), or
// a refined box resting on the floor
struct DomKind {
  int periodic, lid;
  double ztop;
};

// cuTensorMapEncodeTiled, from the driver through the runtime's entry-point
// query (no link against the driver library)
using EncodeTiled = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                 const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encode_tiled() {
  static const EncodeTiled fn = [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return (EncodeTiled) nullptr;
    return (EncodeTiled)p;
  }();
  return fn;
}

// Two tensor maps per domain for the FP32 two-cell stencil: a 3-D view of
// the domain's twenty padded field arrays (x: px, y: py, z: twenty times pz)
// with the box of one haloed tile plane, (TILE_X + 4) x (tile height + 4) x 1,
// for the tile heights 8 and 16.  Points outside the view read as zeros.
static_assert(sizeof(CUtensorMap) == 128, "128-byte tensor maps");
cudaError_t make_tensor_maps(const cc_model *m, std::vector<unsigned char> &out, std::string &why) {
  const EncodeTiled enc = encode_tiled();
  if (!enc) {
    why = "cuTensorMapEncodeTiled not available from the driver";
    return cudaErrorSymbolNotFound;
  }
  out.assign((size_t)m->ndom * 2 * sizeof(CUtensorMap), 0);
  for (int d = 0; d < m->ndom; d++) {
    const DomDev &D = m->dom[d].D;
    for (int t = 0; t < 2; t++) {
      const int ty = t == 0 ? 8 : 16;
      CUtensorMap tm;
      const cuuint64_t dims[3] = {(cuuint64_t)D.px, (cuuint64_t)D.py, (cuuint64_t)D.pz * NBUF * NFIELD};
      const cuuint64_t strides[2] = {(cuuint64_t)D.px * sizeof(float), (cuuint64_t)D.plane * sizeof(float)};
      const cuuint32_t box[3] = {(cuuint32_t)(TILE_X + 4), (cuuint32_t)(ty + 4), 1};
      const cuuint32_t es[3] = {1, 1, 1};
      const CUresult r = enc(&tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, D.f[0][0], dims, strides, box, es,
                             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
      if (r != CUDA_SUCCESS) {
        why = "cuTensorMapEncodeTiled failed with " + std::to_string((int)r) + " for domain " + std::to_string(d);
        return cudaErrorInvalidValue;
      }
      std::memcpy(out.data() + (2 * (size_t)d + t) * sizeof(CUtensorMap), &tm, sizeof(CUtensorMap));
    }
  }
  return cudaSuccess;
}

}  // namespace

namespace {

// Creates the model of the given domains (shared by cc_create and the
// refined constructors); a non-empty layout makes it a refined model.
cc_status create_impl(const std::vector<cc_config> &cfgs, const std::vector<DomKind> &kinds, const Layout &lay,
                      int precision, void *stream, cc_model **out) {
  const int n = (int)cfgs.size();
  cc_model *m = new cc_model();
  m->ndom = n;
  m->prec = precision;
  m->esz = precision == CC_FP64 ? 8 : 4;
  m->st = (cudaStream_t)stream;
  m->dom.resize(n);
  m->refined = !lay.level.empty();
  m->dom_level.assign(n, 0);
  m->blk_off.assign(n, {0, 0});
  if (m->refined) {
    m->dom_level = lay.level;
    m->blk_off = lay.off;
    m->lev_box = lay.lev_box;
    m->nlev = lay.level.back() + 1;
    m->lev_first.assign(m->nlev, 0);
    m->lev_count.assign(m->nlev, 0);
    for (int d = n - 1; d >= 0; d--) m->lev_first[lay.level[d]] = d;
    for (int d = 0; d < n; d++) m->lev_count[lay.level[d]]++;
    m->d_xch.assign(m->nlev, nullptr);
    m->nxch.assign(m->nlev, 0);
    m->lset.assign(m->nlev, LinkSet{});
  }
  cudaError_t e = cudaSuccess;
  auto bail = [&](cudaError_t ee, const char *where) {
    std::string msg = std::string(where) + ": " + cudaGetErrorString(ee);
    cc_destroy(m);
    return fail(nullptr, ee == cudaErrorMemoryAllocation ? CC_ENOMEM : CC_ECUDA, msg);
  };
  size_t max_stage = 16;
  if ((e = full_prepare(precision)) != cudaSuccess) return bail(e, "kernel attributes");
  for (int d = 0; d < n; d++) {
    DomHost &H = m->dom[d];
    H.cfg = cfgs[d];
    const cc_config &c = H.cfg;
    DomDev &D = H.D;
    D.nx = c.nx; D.ny = c.ny; D.nz = c.nz;
    D.px = (c.nx + GX + 4 + 7) / 8 * 8; D.py = c.ny + 2 * GH; D.pz = c.nz + 2 * GH;
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
    D.periodic = kinds[d].periodic;
    D.gox = m->blk_off[d][0];
    D.goy = m->blk_off[d][1];
    D.lid = kinds[d].lid;
    D.ztop = kinds[d].ztop;
    if (D.periodic) {
      // the whole block, corners 0 .. n-1
      D.ci0 = 0; D.ci1 = c.nx; D.cj0 = 0; D.cj1 = c.ny; D.ck1 = c.nz; D.qi0 = 0; D.qj0 = 0;
    } else {
      // a box integrates its cells -2 .. n+1 (k < nz+2) and corners -1 .. n+1
      D.ci0 = -2; D.ci1 = c.nx + 2; D.cj0 = -2; D.cj1 = c.ny + 2; D.ck1 = c.nz + 2; D.qi0 = -1; D.qj0 = -1;
    }
    long long ncol = (long long)c.nx * c.ny, ncell = ncol * c.nz, npc = D.plane;
    // the twenty field arrays back to back, level b field f at
    // (b NFIELD + f) ncellp elements, so that one tensor map covers them
    unsigned char *fields = nullptr;
    if ((e = dalloc(H.allocs, &fields, (size_t)NBUF * NFIELD * D.ncellp * m->esz, m->st)) != cudaSuccess)
      return bail(e, "field alloc");
    for (int b = 0; b < NBUF; b++) {
      for (int f = 0; f < NFIELD; f++) D.f[b][f] = fields + ((size_t)b * NFIELD + f) * D.ncellp * m->esz;
      if ((e = dalloc(H.allocs, &D.ub[b], 3 * npc * m->esz, m->st)) != cudaSuccess) return bail(e, "ub alloc");
    }
    void *bt[7];
    for (int a = 0; a < 7; a++)
      if ((e = dalloc(H.allocs, &bt[a], (size_t)D.pz * m->esz, m->st)) != cudaSuccess) return bail(e, "base alloc");
    D.rhob = bt[0]; D.pb = bt[1]; D.thb = bt[2]; D.pik = bt[3]; D.rhobc = bt[4]; D.tau = bt[5]; D.ipb = bt[6];
    // binomial coefficients C(a, n), n = 1..7, of (1 + x)^a - 1
    for (int w = 0; w < 2; w++) {
      double a = w == 0 ? D.cvcp : D.kap, cn = 1.0;
      float *o = w == 0 ? D.sth : D.sex;
      for (int nn = 1; nn <= 7; nn++) {
        cn = cn * (a - (nn - 1)) / nn;
        o[nn - 1] = (float)cn;
      }
      o[7] = (float)a;
      double *od = w == 0 ? D.dsth : D.dsex;
      cn = 1.0;
      for (int nn = 1; nn <= 12; nn++) {
        cn = cn * (a - (nn - 1)) / nn;
        od[nn - 1] = cn;
      }
      od[12] = a;
    }
    double *h, *vf, *ax, *ay, *az, *ba, *bb, *bn, *mg;
    int8_t *cls, *vcls;
    int32_t *root, *kug, *bK, *bI, *bJ, *mK, *ktop, *kb;
    if ((e = dalloc(H.allocs, &h, ncol * 8, m->st)) ||
        (e = dalloc(H.allocs, &vf, ncell * 8, m->st)) || (e = dalloc(H.allocs, &ax, ncell * 8, m->st)) ||
        (e = dalloc(H.allocs, &ay, ncell * 8, m->st)) ||
        (e = dalloc(H.allocs, &az, ncol * (c.nz + 1) * 8, m->st)) ||
        (e = dalloc(H.allocs, &cls, ncell, m->st)) || (e = dalloc(H.allocs, &root, ncell * 4, m->st)) ||
        (e = dalloc(H.allocs, &kug, npc * 4, m->st)) || (e = dalloc(H.allocs, &vcls, D.ncellp, m->st)) ||
        (e = dalloc(H.allocs, &bK, npc * 4, m->st)) || (e = dalloc(H.allocs, &bI, npc * 4, m->st)) ||
        (e = dalloc(H.allocs, &bJ, npc * 4, m->st)) || (e = dalloc(H.allocs, &ba, npc * 8, m->st)) ||
        (e = dalloc(H.allocs, &bb, npc * 8, m->st)) || (e = dalloc(H.allocs, &bn, 3 * npc * 8, m->st)) ||
        (e = dalloc(H.allocs, &mK, D.ncellp * 4, m->st)) || (e = dalloc(H.allocs, &mg, D.ncellp * 8, m->st)) ||
        (e = dalloc(H.allocs, &ktop, npc * 4, m->st)) || (e = dalloc(H.allocs, &kb, npc * 4, m->st)))
      return bail(e, "geometry alloc");
    DiffCol *dcol;
    if ((e = dalloc(H.allocs, &dcol, npc * sizeof(DiffCol), m->st)) != cudaSuccess) return bail(e, "geometry alloc");
    D.dcol = dcol;
    D.h = h; D.vf = vf; D.ax = ax; D.ay = ay; D.az = az; D.cls = cls; D.root = root; D.kug = kug;
    D.vcls = vcls; D.bK = bK; D.bI = bI; D.bJ = bJ; D.ba = ba; D.bb = bb; D.bn = bn; D.mK = mK; D.mg = mg;
    D.ktop = ktop;
    D.kb = kb;
    if ((e = launch_base(D, precision, c.theta0, c.N, c.p_surf, c.sponge_frac, c.tau_max, m->st)) != cudaSuccess)
      return bail(e, "base state");
    max_stage = std::max(max_stage, (size_t)(ncol * (c.nz + 1 + 2 * HOST_GZ)));
    max_stage = std::max(max_stage, (size_t)(ncol * (c.nz + 1)));
    max_stage = std::max(max_stage, (size_t)(3 * ncol));
  }
  {
    const DomDev &D0 = m->dom[0].D;
    for (int a = 0; a < 8; a++) {
      m->eos.sth[a] = D0.sth[a];
      m->eos.sex[a] = D0.sex[a];
    }
    for (int a = 0; a < 13; a++) {
      m->eos.dsth[a] = D0.dsth[a];
      m->eos.dsex[a] = D0.dsex[a];
    }
    m->eos.p0 = D0.p0;
    m->eos.p0R = D0.p0 / D0.R;
    m->eos.cvcp = D0.cvcp;
    m->eos.kap = D0.kap;
  }
  // TMA tensor maps of the FP32 stencil
  if (precision == CC_FP32) {
    std::vector<unsigned char> maps;
    std::string why;
    if ((e = make_tensor_maps(m, maps, why)) != cudaSuccess) {
      cc_destroy(m);
      return fail(nullptr, CC_ECUDA, "tensor maps: " + why);
    }
    if ((e = dalloc(m->allocs, &m->d_tmaps, maps.size(), m->st)) != cudaSuccess) return bail(e, "tensor maps");
    if ((e = cudaMemcpyAsync(m->d_tmaps, maps.data(), maps.size(), cudaMemcpyHostToDevice, m->st)) != cudaSuccess)
      return bail(e, "tensor map copy");
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
  // (domain, tile, z-chunk) work lists of the full-cell stencil over each
  // domain's computed region, one per schedule (tile height, items per
  // launch): z is split so that every SM gets several work items per launch
  // (all domains of an ensemble share one launch, each level of a refined
  // model, all its blocks, has its own)
  {
    std::vector<ColItem> cols;
    for (int sc = 0; sc < NSCHED; sc++) {
      const int TY = sched_tile_y(precision, sc);
      auto tiles_of = [&](const DomDev &D) {
        return (long long)((D.ci1 - D.ci0 + 3 + TILE_X - 1) / TILE_X) * ((D.cj1 - D.cj0 + TY - 1) / TY);
      };
      long long all_tiles = 0;
      for (auto &H : m->dom) all_tiles += tiles_of(H.D);
      // the tiles that share a launch with domain d
      auto launch_tiles = [&](int d) {
        if (!m->refined) return all_tiles;
        long long t = 0;
        const int l = m->dom_level[d];
        for (int q = m->lev_first[l]; q < m->lev_first[l] + m->lev_count[l]; q++) t += tiles_of(m->dom[q].D);
        return t;
      };
      const long long want = SCHED_ITEMS[sc];
      std::vector<WorkItem> items;
      // FP32: the tiles of a periodic domain go to the second part, gathered
      // from cyclic indices; those of a refined box, whose halos never wrap,
      // to the first, staged with TMA boxes (a domain's tiles stay together,
      // so that neighbouring tiles, which share halo rows in L2, run together)
      const bool split = precision == CC_FP32;
      auto wraps = [&](const DomDev &D, int, int) { return split && D.periodic; };
      for (int part = 0; part < 2; part++) {
        for (int d = 0; d < n; d++) {
          DomHost &H = m->dom[d];
          const DomDev &D = H.D;
          long long tiles = launch_tiles(d);
          long long splits = std::max(1LL, (want + tiles - 1) / tiles);
          int chunk = (int)std::max(8LL, (D.ck1 + splits - 1) / splits);
          (part == 0 ? H.item0 : H.witem0)[sc] = (int)items.size();
          // tiles start at multiples of 4 in x (16-byte halo rows, 16-byte
          // aligned TMA boxes)
          const int ib = D.ci0 - ((D.ci0 % 4) + 4) % 4;
          for (int k0 = 0; k0 < D.ck1; k0 += chunk)
            for (int j0 = D.cj0; j0 < D.cj1; j0 += TY)
              for (int i0 = ib; i0 < D.ci1; i0 += TILE_X) {
                if (wraps(D, i0, j0) != (part == 1)) continue;
                WorkItem w{};
                w.dom = d; w.i0 = i0; w.j0 = j0; w.k0 = k0; w.k1 = std::min(D.ck1, k0 + chunk);
                items.push_back(w);
              }
          (part == 0 ? H.nitem : H.nwitem)[sc] = (int)items.size() - (part == 0 ? H.item0 : H.witem0)[sc];
        }
        (part == 0 ? m->nitems : m->nwitems)[sc] = (int)items.size() - (part == 0 ? 0 : m->nitems[sc]);
      }
      if ((e = dalloc(m->allocs, &m->d_items[sc], sizeof(WorkItem) * items.size(), m->st)) != cudaSuccess)
        return bail(e, "work list");
      if ((e = cudaMemcpyAsync(m->d_items[sc], items.data(), sizeof(WorkItem) * items.size(),
                               cudaMemcpyHostToDevice, m->st)) != cudaSuccess)
        return bail(e, "work list copy");
      if ((e = cudaStreamSynchronize(m->st)) != cudaSuccess) return bail(e, "sync");
    }
    for (int d = 0; d < n; d++) {
      DomHost &H = m->dom[d];
      const DomDev &D = H.D;
      H.col0 = (int)cols.size();
      for (int J = D.qj0; J < D.cj1; J++)
        for (int I = D.qi0; I < D.ci1; I++) cols.push_back(ColItem{d, I, J, 0});
      H.ncol = (int)cols.size() - H.col0;
    }
    m->ncols = (int)cols.size();
    if ((e = dalloc(m->allocs, &m->d_cols, sizeof(ColItem) * cols.size(), m->st)) != cudaSuccess)
      return bail(e, "column list");
    if ((e = cudaMemcpyAsync(m->d_cols, cols.data(), sizeof(ColItem) * cols.size(), cudaMemcpyHostToDevice,
                             m->st)) != cudaSuccess)
      return bail(e, "column list copy");
    if ((e = cudaStreamSynchronize(m->st)) != cudaSuccess) return bail(e, "sync");
  }
  // coarse-fine links of a refined model, one per domain of level >= 1, and
  // the same-level copies of every level made of sibling blocks
  if (m->refined) {
    m->link.resize(n);
    std::vector<std::vector<XchItem>> xch(m->nlev);
    for (int d = 0; d < n; d++) {
      const int lev = m->dom_level[d];
      if (lev == 0) continue;
      LinkHost &K = m->link[d];
      K.box = lay.box[d];
      K.dc = m->lev_first[lev - 1];
      const DomDev &C = m->dom[K.dc].D, &F = m->dom[d].D;
      const cc_box &b = K.box, &U = m->lev_box[lev];
      const int bx = m->blk_off[d][0], by = m->blk_off[d][1];
      K.x0 = b.ox / 2; K.x1 = (b.ox + b.nx) / 2;
      K.y0 = b.oy / 2; K.y1 = (b.oy + b.ny) / 2;
      K.z1 = b.nz / 2;
      // the level's whole box in coarse cells: its outer boundary is the
      // coarse-fine interface (the faces between siblings are not)
      const int ux0 = U.ox / 2, ux1 = (U.ox + U.nx) / 2, uy0 = U.oy / 2, uy1 = (U.oy + U.ny) / 2;
      const bool xlo = bx == 0, xhi = bx + F.nx == U.nx, ylo = by == 0, yhi = by + F.ny == U.ny;
      // The undivided level integrates its cells -2 .. N+1 and corners
      // -1 .. N+1 in x and y below level nz + 2 (the ghost layers included),
      // and every block integrates its own share of them: the point's owner is
      // the block that holds it once clamped into the level's box.  A point
      // of this block's ghost shell within two of its interior (the reach of
      // the stencils of its own points) that the level integrates and another
      // block owns is copied from the owner after every step; a point outside
      // the level's box is injected from the coarser level at every coarse
      // step, as for the undivided level (the ghost layers are both).  The
      // block also integrates the ghost points that siblings own, from shell
      // values it does not keep current; the copies replace those results.
      const int NX = U.nx, NY = U.ny;
      // the copy records hold 32-bit offsets and 16-bit domain indices
      if (m->lev_count[lev] > 1 && (F.ncellp >= (1LL << 31) || n >= 65535)) {
        cc_destroy(m);
        return fail(nullptr, CC_EINVAL, "a block of a cut level is too large for 32-bit offsets");
      }
      auto owner = [&](int gx, int gy) {
        const int cx = std::min(std::max(gx, 0), NX - 1), cy = std::min(std::max(gy, 0), NY - 1);
        for (int q = m->lev_first[lev]; q < m->lev_first[lev] + m->lev_count[lev]; q++) {
          const int ox = m->blk_off[q][0], oy = m->blk_off[q][1];
          const DomDev &Q = m->dom[q].D;
          if (cx >= ox && cx < ox + Q.nx && cy >= oy && cy < oy + Q.ny) return q;
        }
        return d;
      };
      auto copy_from = [&](int q, int i, int j, int k, int kind) {
        const DomDev &Q = m->dom[q].D;
        const int qi = bx + i - m->blk_off[q][0], qj = by + j - m->blk_off[q][1];
        XchItem x{};
        x.ddom = (uint16_t)d; x.sdom = (uint16_t)q; x.kind = kind;
        x.dst = (int32_t)(kind == XCH_COLUMN ? qidx(F, i, j) : pidx(F, i, j, k));
        x.src = (int32_t)(kind == XCH_COLUMN ? qidx(Q, qi, qj) : pidx(Q, qi, qj, k));
        xch[lev].push_back(x);
      };
      std::vector<long long> pcell, pcorn, rcell, rcorn;
      for (int k = -GH; k < F.nz + GH; k++)
        for (int j = -GH; j < F.ny + GH; j++)
          for (int i = -GH; i < F.nx + GH; i++) {
            if (i >= 0 && i < F.nx && j >= 0 && j < F.ny && k < F.nz) continue;
            const int gx = bx + i, gy = by + j;
            const bool inside = gx >= 0 && gx < NX && gy >= 0 && gy < NY && k < F.nz;
            if (!inside && k >= 0) pcell.push_back(pidx(F, i, j, k));
            const bool reach = i >= -2 && i < F.nx + 2 && j >= -2 && j < F.ny + 2;
            if (reach && gx >= -2 && gx < NX + 2 && gy >= -2 && gy < NY + 2 && k >= 0 && k < F.nz + 2) {
              const int q = owner(gx, gy);
              if (q != d) copy_from(q, i, j, k, XCH_CELL);
            }
          }
      for (int Kk = -GH + 1; Kk < F.nz + GH; Kk++)
        for (int J = -GH; J < F.ny + GH; J++)
          for (int I = -GH; I < F.nx + GH; I++) {
            if (I >= 0 && I <= F.nx && J >= 0 && J <= F.ny && Kk <= F.nz) continue;
            const int gx = bx + I, gy = by + J;
            const bool inside = gx >= 0 && gx <= NX && gy >= 0 && gy <= NY && Kk <= F.nz;
            if (!inside) pcorn.push_back(pidx(F, I, J, Kk));
            const bool reach = I >= -2 && I <= F.nx + 2 && J >= -2 && J <= F.ny + 2;
            if (reach && gx >= -1 && gx < NX + 2 && gy >= -1 && gy < NY + 2 && Kk < F.nz + 2) {
              const int q = owner(gx, gy);
              if (q != d) copy_from(q, I, J, Kk, XCH_CORNER);
            }
          }
      for (int J = -GH; J < F.ny + GH; J++)
        for (int I = -GH; I < F.nx + GH; I++) {
          if (I >= 0 && I <= F.nx && J >= 0 && J <= F.ny) continue;
          const int gx = bx + I, gy = by + J;
          const bool reach = I >= -2 && I <= F.nx + 2 && J >= -2 && J <= F.ny + 2;
          if (reach && gx >= -1 && gx < NX + 2 && gy >= -1 && gy < NY + 2) {
            const int q = owner(gx, gy);
            if (q != d) copy_from(q, I, J, 0, XCH_COLUMN);
          }
        }
      // restriction: the coarse cells and corners of this domain within GH
      // of the level's outer boundary (a corner on a cut between siblings
      // belongs to the block on its high side)
      for (int kc = 0; kc < K.z1; kc++)
        for (int jc = K.y0; jc < K.y1; jc++)
          for (int ic = K.x0; ic < K.x1; ic++) {
            int dd = std::min({ic - ux0, ux1 - 1 - ic, jc - uy0, uy1 - 1 - jc, K.z1 - 1 - kc});
            if (dd < GH) rcell.push_back(pidx(C, ic, jc, kc));
          }
      for (int Kc = 1; Kc <= K.z1; Kc++)
        for (int Jc = K.y0; Jc <= K.y1 - (yhi ? 0 : 1); Jc++)
          for (int Ic = K.x0; Ic <= K.x1 - (xhi ? 0 : 1); Ic++) {
            int dd = std::min({Ic - ux0, ux1 - Ic, Jc - uy0, uy1 - Jc, K.z1 - Kc});
            if (dd <= GH) rcorn.push_back(pidx(C, Ic, Jc, Kc));
          }
      std::vector<IfaceFace> faces;
      std::vector<IfaceCell> icells;
      std::map<long long, int> where;
      auto touch = [&](int ci, int cj, int ck, int slot, int q) {
        long long key = pidx(C, ci, cj, ck);
        auto it = where.find(key);
        if (it == where.end()) {
          IfaceCell ic{};
          ic.i = ci; ic.j = cj; ic.k = ck;
          for (int a = 0; a < 6; a++) ic.slot[a] = -1;
          it = where.emplace(key, (int)icells.size()).first;
          icells.push_back(ic);
        }
        icells[it->second].slot[slot] = q;
      };
      // face of axis ax between coarse cells lo (below) and hi (above)
      auto add = [&](int ax, int fi, int fj, int fk, int hi_i, int hi_j, int hi_k) {
        int q = (int)faces.size();
        faces.push_back(IfaceFace{ax, fi, fj, fk});
        int lo_i = hi_i - (ax == 0), lo_j = hi_j - (ax == 1), lo_k = hi_k - (ax == 2);
        touch(lo_i, lo_j, lo_k, ax * 2 + 1, q);
        touch(hi_i, hi_j, hi_k, ax * 2 + 0, q);
      };
      // (only the faces on the level's outer boundary)
      for (int sd = 0; sd < 2; sd++)
        if (sd ? xhi : xlo)
          for (int kc = 0; kc < K.z1; kc++)
            for (int jc = K.y0; jc < K.y1; jc++)
              add(0, sd ? b.nx : 0, 2 * jc - b.oy, 2 * kc, sd ? K.x1 : K.x0, jc, kc);
      for (int sd = 0; sd < 2; sd++)
        if (sd ? yhi : ylo)
          for (int kc = 0; kc < K.z1; kc++)
            for (int ic = K.x0; ic < K.x1; ic++)
              add(1, 2 * ic - b.ox, sd ? b.ny : 0, 2 * kc, ic, sd ? K.y1 : K.y0, kc);
      for (int jc = K.y0; jc < K.y1; jc++)
        for (int ic = K.x0; ic < K.x1; ic++) add(2, 2 * ic - b.ox, 2 * jc - b.oy, b.nz, ic, jc, K.z1);
      LevelLink &L = K.L;
      L.dc = m->d_doms + K.dc;
      L.df = m->d_doms + d;
      L.ox = b.ox;
      L.oy = b.oy;
      auto up = [&](auto &vec, auto **dst) -> cudaError_t {
        using E = typename std::remove_reference<decltype(vec)>::type::value_type;
        E *p = nullptr;
        cudaError_t ee = dalloc(m->allocs, &p, sizeof(E) * vec.size(), m->st);
        if (ee != cudaSuccess) return ee;
        if (!vec.empty())
          ee = cudaMemcpyAsync(p, vec.data(), sizeof(E) * vec.size(), cudaMemcpyHostToDevice, m->st);
        *dst = p;
        return ee;
      };
      const long long *pc = nullptr, *pq = nullptr, *rc = nullptr, *rq = nullptr;
      const IfaceFace *fp = nullptr;
      const IfaceCell *cp = nullptr;
      if ((e = up(pcell, &pc)) || (e = up(pcorn, &pq)) || (e = up(rcell, &rc)) || (e = up(rcorn, &rq)) ||
          (e = up(faces, &fp)) || (e = up(icells, &cp)))
        return bail(e, "refinement lists");
      L.pcell = pc; L.npcell = (long long)pcell.size();
      L.pcorn = pq; L.npcorn = (long long)pcorn.size();
      L.rcell = rc; L.nrcell = (long long)rcell.size();
      L.rcorn = rq; L.nrcorn = (long long)rcorn.size();
      L.faces = fp; L.nfaces = (int)faces.size();
      L.icells = cp; L.nicells = (int)icells.size();
      if ((e = dalloc(m->allocs, &L.regm, faces.size() * m->esz, m->st)) ||
          (e = dalloc(m->allocs, &L.regh, faces.size() * m->esz, m->st)))
        return bail(e, "flux register");
      if ((e = cudaStreamSynchronize(m->st)) != cudaSuccess) return bail(e, "sync");
    }
    for (int l = 0; l < m->nlev; l++) {
      if (xch[l].empty()) continue;
      if ((e = dalloc(m->allocs, &m->d_xch[l], sizeof(XchItem) * xch[l].size(), m->st)) != cudaSuccess ||
          (e = cudaMemcpyAsync(m->d_xch[l], xch[l].data(), sizeof(XchItem) * xch[l].size(), cudaMemcpyHostToDevice,
                               m->st)) != cudaSuccess ||
          (e = cudaStreamSynchronize(m->st)) != cudaSuccess)
        return bail(e, "same-level copies");
      m->nxch[l] = (long long)xch[l].size();
    }
    for (int l = 1; l < m->nlev; l++) {
      std::vector<LevelLink> ls;
      LinkSet &S = m->lset[l];
      for (int d = m->lev_first[l]; d < m->lev_first[l] + m->lev_count[l]; d++) {
        const LevelLink &L = m->link[d].L;
        ls.push_back(L);
        S.maxp = std::max(S.maxp, L.npcell + L.npcorn);
        S.maxr = std::max(S.maxr, L.nrcell + L.nrcorn);
        S.maxf = std::max(S.maxf, (long long)L.nfaces);
        S.maxi = std::max(S.maxi, (long long)L.nicells);
      }
      LevelLink *dl = nullptr;
      if ((e = dalloc(m->allocs, &dl, sizeof(LevelLink) * ls.size(), m->st)) != cudaSuccess ||
          (e = cudaMemcpyAsync(dl, ls.data(), sizeof(LevelLink) * ls.size(), cudaMemcpyHostToDevice, m->st)) !=
              cudaSuccess ||
          (e = cudaStreamSynchronize(m->st)) != cudaSuccess)
        return bail(e, "link sets");
      S.links = dl;
      S.n = (int)ls.size();
    }
  }
  if ((e = dalloc(m->allocs, &m->d_diag, sizeof(double) * (8 + 7 * 256), m->st)) != cudaSuccess) return bail(e, "diag");
  if ((e = dalloc(m->allocs, &m->d_stage, sizeof(double) * max_stage, m->st)) != cudaSuccess) return bail(e, "stage");
  m->stage_elems = max_stage;
  if ((e = dalloc(m->allocs, &m->d_err, sizeof(int), m->st)) != cudaSuccess) return bail(e, "err flag");
  if ((e = dalloc(m->allocs, &m->d_watch, 16, m->st)) != cudaSuccess) return bail(e, "watchdog flag");
  if ((e = cudaMemsetAsync(m->d_watch, 0, 16, m->st)) != cudaSuccess) return bail(e, "watchdog flag");
  if ((e = cudaMallocHost(&m->h_watch, 16)) != cudaSuccess) return bail(e, "watchdog flag");
  *m->h_watch = 0;
  if ((e = cudaEventCreateWithFlags(&m->ev_watch, cudaEventDisableTiming)) != cudaSuccess)
    return bail(e, "watchdog event");
  if ((e = cudaStreamSynchronize(m->st)) != cudaSuccess) return bail(e, "sync");
  *out = m;
  return CC_OK;
}

}  // namespace

extern "C" {

cc_status cc_create(const cc_config *cfgs, int n, int precision, void *stream, cc_model **out) {
  if (!out) return fail(nullptr, CC_EINVAL, "out is NULL");
  *out = nullptr;
  if (!cfgs || n <= 0) return fail(nullptr, CC_EINVAL, "need at least one domain");
  if (precision != CC_FP64 && precision != CC_FP32) return fail(nullptr, CC_EINVAL, "precision must be CC_FP64 or CC_FP32");
  std::vector<cc_config> cv(cfgs, cfgs + n);
  std::vector<DomKind> kinds(n);
  for (int d = 0; d < n; d++) {
    std::string why;
    if (!valid_cfg(cfgs[d], why)) return fail(nullptr, CC_EINVAL, "domain " + std::to_string(d) + ": " + why);
    if (cfgs[d].R != cfgs[0].R || cfgs[d].cp != cfgs[0].cp || cfgs[d].p0 != cfgs[0].p0)
      return fail(nullptr, CC_EINVAL, "all domains of a model share R, cp and p0");
    kinds[d] = DomKind{1, 1, cfgs[d].nz * cfgs[d].dz};
  }
  return create_impl(cv, kinds, Layout{}, precision, stream, out);
}

cc_status cc_create_refined(const cc_config *base, int nlev, const cc_box *boxes, int precision, void *stream,
                            cc_model **out) {
  return cc_create_refined_blocks(base, nlev, boxes, 0, nullptr, 0, nullptr, precision, stream, out);
}

cc_status cc_create_refined_blocks(const cc_config *base, int nlev, const cc_box *boxes, int nxcut,
                                   const int *xcut, int nycut, const int *ycut, int precision, void *stream,
                                   cc_model **out) {
  if (!out) return fail(nullptr, CC_EINVAL, "out is NULL");
  *out = nullptr;
  if (!base || !boxes) return fail(nullptr, CC_EINVAL, "null argument");
  if (nxcut < 0 || nycut < 0 || (nxcut > 0 && !xcut) || (nycut > 0 && !ycut))
    return fail(nullptr, CC_EINVAL, "bad cut lists");
  if (nlev < 2 || nlev > 8) return fail(nullptr, CC_EINVAL, "nlev must be 2 .. 8");
  if (precision != CC_FP64 && precision != CC_FP32) return fail(nullptr, CC_EINVAL, "precision must be CC_FP64 or CC_FP32");
  std::string why;
  if (!valid_cfg(*base, why)) return fail(nullptr, CC_EINVAL, "level 0: " + why);
  std::vector<cc_config> cv(nlev);
  std::vector<DomKind> kinds(nlev);
  std::vector<cc_box> bx(boxes, boxes + nlev - 1);
  const double ztop = base->nz * base->dz;
  cv[0] = *base;
  kinds[0] = DomKind{1, 1, ztop};
  for (int l = 1; l < nlev; l++) {
    const cc_box &b = bx[l - 1];
    const cc_config &c = cv[l - 1];
    int x0 = b.ox / 2, x1 = (b.ox + b.nx) / 2, y0 = b.oy / 2, y1 = (b.oy + b.ny) / 2, z1 = b.nz / 2;
    if (((b.ox | b.oy | b.nx | b.ny | b.nz) & 1) || b.nx <= 0 || b.ny <= 0 || b.nz <= 0)
      return fail(nullptr, CC_EINVAL, "box " + std::to_string(l) + ": extents and offsets must be even and positive");
    if (x0 < 8 || y0 < 8 || x1 > c.nx - 8 || y1 > c.ny - 8 || z1 > c.nz - 8)
      return fail(nullptr, CC_EINVAL,
                  "box " + std::to_string(l) + ": covered box must lie 8 cells inside the coarser level");
    if (b.nx <= 2 * FLAT_MARGIN || b.ny <= 2 * FLAT_MARGIN)
      return fail(nullptr, CC_EINVAL, "box " + std::to_string(l) + ": nx and ny must exceed 16");
    cc_config f = *base;
    double s = std::ldexp(1.0, -l);
    f.nx = b.nx; f.ny = b.ny; f.nz = b.nz;
    f.dx = base->dx * s; f.dy = base->dy * s; f.dz = base->dz * s; f.dt = base->dt * s;
    if (!valid_cfg(f, why)) return fail(nullptr, CC_EINVAL, "level " + std::to_string(l) + ": " + why);
    cv[l] = f;
    kinds[l] = DomKind{0, 0, ztop};
  }
  // the finest level's blocks: cut positions (even, increasing, every block
  // wider than twice the flat margin), blocks by y, then x
  const cc_box &fb = bx[nlev - 2];
  std::vector<int> xs{0}, ys{0};
  for (int a = 0; a < nxcut; a++) xs.push_back(xcut[a]);
  for (int a = 0; a < nycut; a++) ys.push_back(ycut[a]);
  xs.push_back(fb.nx);
  ys.push_back(fb.ny);
  for (size_t a = 1; a < xs.size(); a++)
    if ((xs[a] & 1) || xs[a] - xs[a - 1] <= 2 * FLAT_MARGIN + 1)
      return fail(nullptr, CC_EINVAL, "x cuts must be even, increasing and leave blocks of at least 18 cells");
  for (size_t a = 1; a < ys.size(); a++)
    if ((ys[a] & 1) || ys[a] - ys[a - 1] <= 2 * FLAT_MARGIN + 1)
      return fail(nullptr, CC_EINVAL, "y cuts must be even, increasing and leave blocks of at least 18 cells");
  Layout lay;
  lay.lev_box.assign(nlev, cc_box{});
  for (int l = 1; l < nlev; l++) lay.lev_box[l] = bx[l - 1];
  std::vector<cc_config> cvb(cv.begin(), cv.end() - 1);
  std::vector<DomKind> kb(kinds.begin(), kinds.end() - 1);
  for (int l = 0; l < nlev - 1; l++) {
    lay.level.push_back(l);
    lay.box.push_back(l ? bx[l - 1] : cc_box{});
    lay.off.push_back({0, 0});
  }
  for (size_t by = 0; by + 1 < ys.size(); by++)
    for (size_t bxi = 0; bxi + 1 < xs.size(); bxi++) {
      cc_config f = cv[nlev - 1];
      f.nx = xs[bxi + 1] - xs[bxi];
      f.ny = ys[by + 1] - ys[by];
      cc_box b = fb;
      b.ox = fb.ox + xs[bxi];
      b.oy = fb.oy + ys[by];
      b.nx = f.nx;
      b.ny = f.ny;
      cvb.push_back(f);
      kb.push_back(kinds[nlev - 1]);
      lay.level.push_back(nlev - 1);
      lay.box.push_back(b);
      lay.off.push_back({xs[bxi], ys[by]});
    }
  return create_impl(cvb, kb, lay, precision, stream, out);
}

cc_status cc_domain_block(const cc_model *m, int d, int *level, int *ox, int *oy) {
  if (!m) return fail(nullptr, CC_EINVAL, "null model");
  if (d < 0 || d >= m->ndom) return fail(const_cast<cc_model *>(m), CC_EINVAL, "domain index out of range");
  if (level) *level = m->dom_level[d];
  if (ox) *ox = m->blk_off[d][0];
  if (oy) *oy = m->blk_off[d][1];
  return CC_OK;
}

int cc_domain_count(const cc_model *m) { return m ? m->ndom : 0; }

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
  for (auto &g : m->graphs) cudaGraphExecDestroy(g.exec);
  if (m->cap) cudaStreamDestroy(m->cap);
  if (m->xs) {
    cudaStreamSynchronize(m->xs);
    cudaStreamDestroy(m->xs);
  }
  for (int a = 0; a < 2; a++) {
    if (m->ev_copied[a]) cudaEventDestroy(m->ev_copied[a]);
    if (m->ev_staged[a]) cudaEventDestroy(m->ev_staged[a]);
  }
  cudaFree(m->d_stage2);
  for (auto e : m->ev_bulk) cudaEventDestroy(e);
  if (m->ev_bulk_done) cudaEventDestroy(m->ev_bulk_done);
  cudaFree(m->d_bulk);
  if (m->h_watch) cudaFreeHost(m->h_watch);
  if (m->ev_watch) cudaEventDestroy(m->ev_watch);
  delete m;
  return CC_OK;
}

const char *cc_last_error(const cc_model *m) {
  if (!m) return g_create_error.c_str();
  return m->err.c_str();
}

// The heights every terrain must satisfy: finite, >= 0, below the top; a
// box level flat within FLAT_MARGIN corners of its edges.
static cc_status check_terrain(cc_model *m, const DomHost &H, const double *corner_h) {
  const int nx = H.cfg.nx, ny = H.cfg.ny;
  long long ncol = (long long)nx * ny;
  double top = H.cfg.nz * H.cfg.dz;
  for (long long q = 0; q < ncol; q++) {
    double v = corner_h[q];
    if (!std::isfinite(v) || v < 0.0 || v >= top)
      return fail(m, CC_EINVAL, "terrain heights must be finite, >= 0 and below the top");
  }
  if (!H.D.periodic) {
    for (int J = 0; J < ny; J++)
      for (int I = 0; I < nx; I++) {
        bool edge = I <= FLAT_MARGIN || J <= FLAT_MARGIN || I >= nx - FLAT_MARGIN || J >= ny - FLAT_MARGIN;
        if (edge && corner_h[(long long)J * nx + I] != 0.0)
          return fail(m, CC_EINVAL, "terrain of a refined box must be zero within 8 corners of its edges");
      }
  }
  return CC_OK;
}

cc_status cc_set_terrain(cc_model *m, int d, const double *corner_h) {
  if (!m || !corner_h) return fail(m, CC_EINVAL, "null argument");
  if (d < 0 || d >= m->ndom) return fail(m, CC_EINVAL, "domain index out of range");
  DomHost &H = m->dom[d];
  long long ncol = (long long)H.cfg.nx * H.cfg.ny;
  cc_status r = check_terrain(m, H, corner_h);
  if (r != CC_OK) return r;
  CK(m, cudaMemcpyAsync((void *)H.D.h, corner_h, ncol * 8, cudaMemcpyHostToDevice, m->st), "terrain copy");
  CK(m, cudaStreamSynchronize(m->st), "terrain sync");
  H.hh.assign(corner_h, corner_h + ncol);
  H.terrain = true;
  m->geom = false;
  m->state = false;
  return CC_OK;
}

cc_status cc_set_terrain_analytic(cc_model *m, int d, int kind, const double *params) {
  if (!m || !params) return fail(m, CC_EINVAL, "null argument");
  if (d < 0 || d >= m->ndom) return fail(m, CC_EINVAL, "domain index out of range");
  if (kind < CC_HILL_BELL || kind > CC_HILL_COSINE) return fail(m, CC_EINVAL, "unknown hill kind");
  for (int a = 0; a < 4; a++)
    if (!std::isfinite(params[a])) return fail(m, CC_EINVAL, "non-finite hill parameter");
  if (params[0] < 0.0 || params[1] <= 0.0) return fail(m, CC_EINVAL, "hill height < 0 or width <= 0");
  DomHost &H = m->dom[d];
  long long ncol = (long long)H.cfg.nx * H.cfg.ny;
  H.terrain = false;
  m->geom = false;
  m->state = false;
  CK(m, launch_hill((double *)H.D.h, H.cfg.nx, H.cfg.ny, H.cfg.dx, H.cfg.dy, kind, params[0], params[1], params[2],
                    params[3], m->st), "hill");
  std::vector<double> hh(ncol);
  CK(m, cudaMemcpyAsync(hh.data(), H.D.h, ncol * 8, cudaMemcpyDeviceToHost, m->st), "hill copy");
  CK(m, cudaStreamSynchronize(m->st), "hill sync");
  cc_status r = check_terrain(m, H, hh.data());
  if (r != CC_OK) return r;
  H.hh.swap(hh);
  H.terrain = true;
  return CC_OK;
}

cc_status cc_get_terrain(const cc_model *mc, int d, double *corner_h) {
  cc_model *m = const_cast<cc_model *>(mc);
  if (!m || !corner_h) return fail(m, CC_EINVAL, "null argument");
  if (d < 0 || d >= m->ndom) return fail(m, CC_EINVAL, "domain index out of range");
  const DomHost &H = m->dom[d];
  if (!H.terrain) return fail(m, CC_ESTATE, "terrain not set");
  std::memcpy(corner_h, H.hh.data(), H.hh.size() * sizeof(double));
  return CC_OK;
}

cc_status cc_build_geometry(cc_model *m) {
  if (!m) return fail(m, CC_EINVAL, "null model");
  for (auto &H : m->dom)
    if (!H.terrain) return fail(m, CC_ESTATE, "terrain not set for every domain");
  // a coarser level is flat around every covered box: the coarse cells that
  // exchange fluxes with the box are full cells
  for (int l = 1; l < m->nlev; l++) {
    const cc_box &U = m->lev_box[l];
    const DomHost &C = m->dom[m->lev_first[l - 1]];
    for (int J = U.oy / 2 - 4; J <= (U.oy + U.ny) / 2 + 4; J++)
      for (int I = U.ox / 2 - 4; I <= (U.ox + U.nx) / 2 + 4; I++)
        if (C.hh[(long long)wrapi(J, C.cfg.ny) * C.cfg.nx + wrapi(I, C.cfg.nx)] != 0.0)
          return fail(m, CC_EGEOM, "level " + std::to_string(l - 1) +
                                       ": terrain must be flat within 4 cells of the refined box");
  }
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
    if (!H.D.periodic) CK(m, launch_flat_columns(H.D, m->st), "frame columns");
    CK(m, launch_diffcols(H.D, m->st), "diffusion stencils");
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
    H.group0 = (int)all.size();
    H.ngroup = ng;
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
  // interior columns of the padded column arrays
  auto cols = [&](const auto *src, auto *dst, int w, const char *what) -> cc_status {
    using E = typename std::remove_const<typename std::remove_pointer<decltype(src)>::type>::type;
    E *tmp = (E *)m->d_stage;
    k_gather_cols<E><<<nb256(ncol * w), 256, 0, m->st>>>(src, tmp, D, w);
    CK(m, cudaGetLastError(), what);
    CK(m, cudaMemcpyAsync(dst, tmp, ncol * w * sizeof(E), cudaMemcpyDeviceToHost, m->st), what);
    CK(m, cudaStreamSynchronize(m->st), what);
    return CC_OK;
  };
  cc_status r = CC_OK;
  if (bK && (r = cols(D.bK, bK, 1, "bK")) != CC_OK) return r;
  if (bI && (r = cols(D.bI, bI, 1, "bI")) != CC_OK) return r;
  if (bJ && (r = cols(D.bJ, bJ, 1, "bJ")) != CC_OK) return r;
  if (ba && (r = cols(D.ba, ba, 1, "ba")) != CC_OK) return r;
  if (bb && (r = cols(D.bb, bb, 1, "bb")) != CC_OK) return r;
  if (bn && (r = cols(D.bn, bn, 3, "bn")) != CC_OK) return r;
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
      CK(m, cudaMemsetAsync(H.D.ub[b], 0, 3 * (size_t)H.D.plane * m->esz, m->st), "ub reset");
    }
    for (int a = 0; a < 4; a++) H.r[a] = a;
    H.nsteps = 0;
  }
  for (int d = 0; d < m->ndom; d++)
    CK(m, launch_init_momentum(m->dom[d].D, m->d_doms + d, m->prec, m->dom[d].r[1], m->dom[d].cfg.U, m->st),
       "init momentum");
  StepLaunch L = make_launch(m);
  CK(m, launch_diagnose(L, m->prec, 1, 1, 1, 1, 1, 0, m->st), "init diagnose");
  // refined model: fine -> coarse, then coarse -> fine, down the hierarchy,
  // then the same-level copies between the blocks of a level
  for (int l = 1; l < m->nlev; l++) {
    const int d0 = m->lev_first[l], d1 = d0 + m->lev_count[l];
    for (int d = d0; d < d1; d++) {
      const LevelLink &K = m->link[d].L;
      CK(m, cudaMemsetAsync(K.regm, 0, K.nfaces * m->esz, m->st), "register reset");
      CK(m, cudaMemsetAsync(K.regh, 0, K.nfaces * m->esz, m->st), "register reset");
    }
    CK(m, launch_restrict(m->lset[l], m->prec, m->dom[d0].r[1], m->st), "init restrict");
    CK(m, launch_prolong(m->lset[l], m->prec, m->dom[m->lev_first[l - 1]].r[1], m->st), "init prolong");
    CK(m, launch_exchange(m->d_doms, m->d_xch[l], m->nxch[l], m->prec, m->dom[d0].r[0], m->dom[d0].r[1], m->st),
       "init same-level copies");
  }
  cc_status w = watch_reset(m);
  if (w != CC_OK) return w;
  CK(m, cudaStreamSynchronize(m->st), "init sync");
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
  }  // CC_UB: 3 values per column, through the padded column layout
  *nlev = D.nz + 1 + 2 * HOST_GZ;
  *kfirst = -HOST_GZ;
  return ncol * (*nlev);
}

}  // extern "C"

// Transfers through the model's device staging buffer, in the model's
// stream order (the staging buffer is reused only after the previous
// transfer's kernel or copy, so no host wait is needed between them).
// The transfer stream, its events and the second staging buffer, made on
// first use.
static cc_status transfer_setup(cc_model *m) {
  if (m->xs) return CC_OK;
  CK(m, cudaStreamCreateWithFlags(&m->xs, cudaStreamNonBlocking), "transfer stream");
  for (int a = 0; a < 2; a++) {
    CK(m, cudaEventCreateWithFlags(&m->ev_copied[a], cudaEventDisableTiming), "transfer event");
    CK(m, cudaEventCreateWithFlags(&m->ev_staged[a], cudaEventDisableTiming), "transfer event");
  }
  cudaError_t e = cudaMalloc(&m->d_stage2, sizeof(double) * m->stage_elems);
  if (e != cudaSuccess) {
    m->d_stage2 = nullptr;
    return fail(m, e == cudaErrorMemoryAllocation ? CC_ENOMEM : CC_ECUDA, "second staging buffer");
  }
  return CC_OK;
}

// f32: the host buffer holds FP32 values (FP32 models only, where the
// prognostic fields are FP32, so nothing is rounded either way)
static cc_status upload(cc_model *m, int d, int field, int level, const void *host, bool sync, bool f32 = false) {
  if (!m || !host) return fail(m, CC_EINVAL, "null argument");
  if (f32 && m->prec != CC_FP32) return fail(m, CC_EINVAL, "FP32 host buffers need an FP32 model");
  if (d < 0 || d >= m->ndom) return fail(m, CC_EINVAL, "domain index out of range");
  if (field < 0 || field > CC_UB || level < 0 || level > 1) return fail(m, CC_EINVAL, "bad field or level");
  if (!m->state) return fail(m, CC_ESTATE, "state not initialised");
  cc_status r = transfer_setup(m);
  if (r != CC_OK) return r;
  const DomDev &D = m->dom[d].D;
  int buf = level == 0 ? m->dom[d].r[0] : m->dom[d].r[1];
  int nlev, kfirst;
  long long n = field_elems(D, field, &nlev, &kfirst);
  // host -> staging on the transfer stream, once the model's stream is done
  // with this staging buffer; the conversion into the field on the model's
  // stream after the copy
  const int sl = m->xslot;
  m->xslot ^= 1;
  double *stage = sl ? m->d_stage2 : m->d_stage;
  if (m->used_valid[sl]) CK(m, cudaStreamWaitEvent(m->xs, m->ev_staged[sl], 0), "upload order");
  CK(m, cudaMemcpyAsync(stage, host, n * (f32 ? 4 : 8), cudaMemcpyHostToDevice, m->xs), "upload");
  CK(m, cudaEventRecord(m->ev_copied[sl], m->xs), "upload event");
  CK(m, cudaStreamWaitEvent(m->st, m->ev_copied[sl], 0), "upload order");
  const float *stage32 = (const float *)stage;
  if (field == CC_UB) {
    if (m->prec == CC_FP64) k_scatter_cols<double><<<nb256(n), 256, 0, m->st>>>(stage, (double *)D.ub[buf], D, 3);
    else if (f32) k_scatter_cols<float><<<nb256(n), 256, 0, m->st>>>(stage32, (float *)D.ub[buf], D, 3);
    else k_scatter_cols<float><<<nb256(n), 256, 0, m->st>>>(stage, (float *)D.ub[buf], D, 3);
  } else {
    void *dst = D.f[buf][field];
    if (m->prec == CC_FP64) k_scatter<double><<<nb256(n), 256, 0, m->st>>>(stage, (double *)dst, D, nlev, kfirst);
    else if (f32) k_scatter<float><<<nb256(n), 256, 0, m->st>>>(stage32, (float *)dst, D, nlev, kfirst);
    else k_scatter<float><<<nb256(n), 256, 0, m->st>>>(stage, (float *)dst, D, nlev, kfirst);
  }
  CK(m, cudaGetLastError(), "upload scatter");
  CK(m, cudaEventRecord(m->ev_staged[sl], m->st), "upload event");
  m->used_valid[sl] = true;
  if (sync) CK(m, cudaStreamSynchronize(m->st), "upload sync");
  return CC_OK;
}

// elements of the whole two-time-level state in the host layout (five fields,
// levels 0 and 1, every domain)
static long long state_elems(const cc_model *m) {
  long long n = 0;
  int nlev, kfirst;
  for (const auto &H : m->dom)
    for (int f = 0; f < NFIELD; f++) n += 2 * field_elems(H.D, f, &nlev, &kfirst);
  return n;
}

// the whole state from one host buffer: one copy per domain on the transfer
// stream, each domain's conversions on the model's stream once its copy is in
static cc_status upload_all(cc_model *m, const void *host, bool f32) {
  if (!m || !host) return fail(m, CC_EINVAL, "null argument");
  if (f32 && m->prec != CC_FP32) return fail(m, CC_EINVAL, "FP32 host buffers need an FP32 model");
  if (!m->state) return fail(m, CC_ESTATE, "state not initialised");
  cc_status r = transfer_setup(m);
  if (r != CC_OK) return r;
  const size_t es = f32 ? sizeof(float) : sizeof(double);
  const size_t bytes = (size_t)state_elems(m) * es;
  if (m->bulk_bytes < bytes) {
    if (m->d_bulk) {
      // the stream may still read the smaller buffer
      CK(m, cudaStreamSynchronize(m->st), "bulk staging sync");
      cudaFree(m->d_bulk);
      m->d_bulk = nullptr;
      m->bulk_bytes = 0;
    }
    cudaError_t e = cudaMalloc(&m->d_bulk, bytes);
    if (e != cudaSuccess) {
      m->d_bulk = nullptr;
      cudaGetLastError();
      return fail(m, e == cudaErrorMemoryAllocation ? CC_ENOMEM : CC_ECUDA, "whole-state staging buffer");
    }
    m->bulk_bytes = bytes;
  }
  while (m->ev_bulk.size() < m->dom.size()) {
    cudaEvent_t e = nullptr;
    CK(m, cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "transfer event");
    m->ev_bulk.push_back(e);
  }
  if (!m->ev_bulk_done) CK(m, cudaEventCreateWithFlags(&m->ev_bulk_done, cudaEventDisableTiming), "transfer event");
  // the copies overwrite the staging buffer once the previous whole-state
  // upload's conversions have read it
  if (m->bulk_used) CK(m, cudaStreamWaitEvent(m->xs, m->ev_bulk_done, 0), "upload order");
  char *stage = (char *)m->d_bulk;
  const char *src = (const char *)host;
  size_t off = 0;
  for (int d = 0; d < m->ndom; d++) {
    const DomDev &D = m->dom[d].D;
    int nlev, kfirst;
    size_t bd = 0;
    for (int f = 0; f < NFIELD; f++) bd += 2 * (size_t)field_elems(D, f, &nlev, &kfirst) * es;
    CK(m, cudaMemcpyAsync(stage + off, src + off, bd, cudaMemcpyHostToDevice, m->xs), "upload");
    CK(m, cudaEventRecord(m->ev_bulk[d], m->xs), "upload event");
    CK(m, cudaStreamWaitEvent(m->st, m->ev_bulk[d], 0), "upload order");
    for (int f = 0; f < NFIELD; f++)
      for (int level = 0; level < 2; level++) {
        const long long n = field_elems(D, f, &nlev, &kfirst);
        void *dst = D.f[level == 0 ? m->dom[d].r[0] : m->dom[d].r[1]][f];
        const void *a = stage + off;
        if (m->prec == CC_FP64)
          k_scatter<double><<<nb256(n), 256, 0, m->st>>>((const double *)a, (double *)dst, D, nlev, kfirst);
        else if (f32)
          k_scatter<float><<<nb256(n), 256, 0, m->st>>>((const float *)a, (float *)dst, D, nlev, kfirst);
        else
          k_scatter<float><<<nb256(n), 256, 0, m->st>>>((const double *)a, (float *)dst, D, nlev, kfirst);
        off += (size_t)n * es;
      }
  }
  CK(m, cudaGetLastError(), "upload scatter");
  CK(m, cudaEventRecord(m->ev_bulk_done, m->st), "upload event");
  m->bulk_used = true;
  return CC_OK;
}

static cc_status download(cc_model *m, int d, int field, int level, void *host, bool sync, bool f32 = false) {
  if (!m || !host) return fail(m, CC_EINVAL, "null argument");
  if (f32 && m->prec != CC_FP32) return fail(m, CC_EINVAL, "FP32 host buffers need an FP32 model");
  if (d < 0 || d >= m->ndom) return fail(m, CC_EINVAL, "domain index out of range");
  if (field < 0 || field > CC_UB || level < 0 || level > 1) return fail(m, CC_EINVAL, "bad field or level");
  if (!m->state) return fail(m, CC_ESTATE, "state not initialised");
  cc_status r = transfer_setup(m);
  if (r != CC_OK) return r;
  const DomDev &D = m->dom[d].D;
  int buf = level == 0 ? m->dom[d].r[0] : m->dom[d].r[1];
  int nlev, kfirst;
  long long n = field_elems(D, field, &nlev, &kfirst);
  // gather and copy on the model's stream (an upload's copy into this
  // staging buffer is ordered before them by its conversion kernel)
  const int sl = m->xslot;
  m->xslot ^= 1;
  double *stage = sl ? m->d_stage2 : m->d_stage;
  float *stage32 = (float *)stage;
  if (field == CC_UB) {
    if (m->prec == CC_FP64)
      k_gather_cols_cvt<double><<<nb256(n), 256, 0, m->st>>>((const double *)D.ub[buf], stage, D, 3);
    else if (f32)
      k_gather_cols_cvt<float><<<nb256(n), 256, 0, m->st>>>((const float *)D.ub[buf], stage32, D, 3);
    else
      k_gather_cols_cvt<float><<<nb256(n), 256, 0, m->st>>>((const float *)D.ub[buf], stage, D, 3);
  } else {
    const void *src = D.f[buf][field];
    if (m->prec == CC_FP64)
      k_gather<double><<<nb256(n), 256, 0, m->st>>>((const double *)src, stage, D, nlev, kfirst);
    else if (f32)
      k_gather<float><<<nb256(n), 256, 0, m->st>>>((const float *)src, stage32, D, nlev, kfirst);
    else
      k_gather<float><<<nb256(n), 256, 0, m->st>>>((const float *)src, stage, D, nlev, kfirst);
  }
  CK(m, cudaGetLastError(), "download gather");
  CK(m, cudaMemcpyAsync(host, stage, n * (f32 ? 4 : 8), cudaMemcpyDeviceToHost, m->st), "download");
  CK(m, cudaEventRecord(m->ev_staged[sl], m->st), "download event");
  m->used_valid[sl] = true;
  if (sync) CK(m, cudaStreamSynchronize(m->st), "download sync");
  return CC_OK;
}

extern "C" {

cc_status cc_upload_state(cc_model *m, int d, int field, int level, const double *host) {
  return upload(m, d, field, level, host, true);
}

cc_status cc_download_state(const cc_model *m, int d, int field, int level, double *host) {
  return download(const_cast<cc_model *>(m), d, field, level, host, true);
}

cc_status cc_download_derived(const cc_model *mc, int d, int which, int level, double *host) {
  cc_model *m = const_cast<cc_model *>(mc);
  if (!m || !host) return fail(m, CC_EINVAL, "null argument");
  if (d < 0 || d >= m->ndom) return fail(m, CC_EINVAL, "domain index out of range");
  if (which < CC_U || which > CC_THETA_P || level < 0 || level > 1 || (which != CC_THETA_P && level != 1))
    return fail(m, CC_EINVAL, "bad field or level (velocities: level 1 only)");
  if (!m->state) return fail(m, CC_ESTATE, "state not initialised");
  const DomHost &H = m->dom[d];
  const long long n = (long long)H.D.nx * H.D.ny * (which == CC_THETA_P ? H.D.nz : H.D.nz + 1);
  const int buf = level == 0 ? H.r[0] : H.r[1];
  CK(m, launch_derived(H.D, m->d_doms + d, m->prec, buf, which, m->d_stage, m->st), "derived");
  CK(m, cudaMemcpyAsync(host, m->d_stage, n * 8, cudaMemcpyDeviceToHost, m->st), "derived copy");
  CK(m, cudaStreamSynchronize(m->st), "derived sync");
  return CC_OK;
}

cc_status cc_error_norms(const cc_model *ac, int da, const cc_model *bc, int db, int which, double zmin,
                         double *out) {
  cc_model *a = const_cast<cc_model *>(ac), *b = const_cast<cc_model *>(bc);
  if (!a || !b || !out) return fail(a, CC_EINVAL, "null argument");
  if (da < 0 || da >= a->ndom || db < 0 || db >= b->ndom) return fail(a, CC_EINVAL, "domain index out of range");
  if (which < CC_U || which > CC_W) return fail(a, CC_EINVAL, "error norms are of a velocity component");
  if (!std::isfinite(zmin) && !(zmin < 0)) return fail(a, CC_EINVAL, "zmin must be finite or -inf");
  if (!a->state || !b->state) return fail(a, CC_ESTATE, "state not initialised");
  const DomHost &A = a->dom[da], &B = b->dom[db];
  const cc_config &ca = A.cfg, &cb = B.cfg;
  // spacing ratio dx_a / dx_b = p / q in lowest terms, q <= 16
  int p = 0, q = 0;
  for (int qq = 1; qq <= 16 && !p; qq++) {
    const double pp = ca.dx / cb.dx * qq;
    const int pi = (int)std::floor(pp + 0.5);
    if (pi >= qq && std::fabs(pi - pp) <= 1e-9 * pp) { p = pi; q = qq; }
  }
  if (!p || std::fabs(p * cb.dy - q * ca.dy) > 1e-9 * q * ca.dy || std::fabs(p * cb.dz - q * ca.dz) > 1e-9 * q * ca.dz ||
      (long long)ca.nx * p != (long long)cb.nx * q || (long long)ca.ny * p != (long long)cb.ny * q ||
      (long long)ca.nz * p != (long long)cb.nz * q)
    return fail(a, CC_EINVAL, "the second model must refine the first by one ratio p/q (q <= 16) over the same domain");
  int kmin = 0;
  while (kmin <= ca.nz && !(kmin * ca.dz > zmin)) kmin++;
  double h[2] = {0.0, 0.0};
  const long long n = (long long)((ca.nx + q - 1) / q) * ((ca.ny + q - 1) / q) * (ca.nz / q + 1 - (kmin + q - 1) / q);
  if (n > 0) {
    CK(a, cudaStreamSynchronize(b->st), "norms: sync of the finer model");
    CK(a, launch_norms(a->d_doms + da, a->prec, A.r[1], b->d_doms + db, b->prec, B.r[1], which, p, q, kmin, a->d_diag,
                       a->d_diag + 8, a->st), "norms");
    CK(a, cudaMemcpyAsync(h, a->d_diag, sizeof(h), cudaMemcpyDeviceToHost, a->st), "norms copy");
    CK(a, cudaStreamSynchronize(a->st), "norms sync");
  }
  out[0] = n > 0 ? h[0] / n : 0.0;
  out[1] = n > 0 ? std::sqrt(h[1] / n) : 0.0;
  out[2] = (double)n;
  return CC_OK;
}

cc_status cc_upload_state_async(cc_model *m, int d, int field, int level, const double *host) {
  return upload(m, d, field, level, host, false);
}

cc_status cc_download_state_async(const cc_model *m, int d, int field, int level, double *host) {
  return download(const_cast<cc_model *>(m), d, field, level, host, false);
}

cc_status cc_upload_state_f32(cc_model *m, int d, int field, int level, const float *host) {
  return upload(m, d, field, level, host, true, true);
}

cc_status cc_download_state_f32(const cc_model *m, int d, int field, int level, float *host) {
  return download(const_cast<cc_model *>(m), d, field, level, host, true, true);
}

cc_status cc_upload_state_f32_async(cc_model *m, int d, int field, int level, const float *host) {
  return upload(m, d, field, level, host, false, true);
}

cc_status cc_download_state_f32_async(const cc_model *m, int d, int field, int level, float *host) {
  return download(const_cast<cc_model *>(m), d, field, level, host, false, true);
}

cc_status cc_state_elems(const cc_model *m, long long *n) {
  if (!m || !n) return fail(const_cast<cc_model *>(m), CC_EINVAL, "null argument");
  *n = state_elems(m);
  return CC_OK;
}

cc_status cc_upload_all_async(cc_model *m, const double *host) { return upload_all(m, host, false); }

cc_status cc_upload_all_f32_async(cc_model *m, const float *host) { return upload_all(m, host, true); }

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
  if (m->dry) return cudaSuccess;
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

// One step of domain d (every domain of an ensemble when d < 0): the
// full-cell stencil, the cut cells, the coarse cells next to a refined box
// (flux register), then the velocity diagnosis; rotates the roles.
// One step of every domain (lev < 0) or of level lev of a refined model (all
// its blocks), with the flux-register corrections of the next finer level's
// interface cells, then the same-level copies between the level's blocks.
static cc_status step_domains(cc_model *m, int lev, long long &nl) {
  DomHost &H0 = m->dom[lev < 0 ? 0 : m->lev_first[lev]];
  const int first = H0.nsteps == 0;
  const int rO = first ? H0.r[1] : H0.r[0];
  const int rC = H0.r[1], rN = H0.r[2], rF = H0.r[3], pr = m->prec;
  cudaStream_t st = m->st;
  StepLaunch L = make_launch(m, lev);
  if (L.nitems > 0 || L.nwitems > 0) {
    CK(m, timed(m, CC_K_FULL, [&] { return launch_full(L, pr, rO, rC, rN, rF, first, st); }), "full-cell stencil");
    nl += (L.nitems > 0) + (L.nwitems > 0);
  }
  if (L.ngroups > 0) {
    CK(m, timed(m, CC_K_GROUPS, [&] { return launch_groups(L, pr, rO, rC, rN, rF, first, st); }), "cut cells");
    nl++;
  }
  if (lev >= 0 && lev + 1 < m->nlev) {
    const LinkSet &S = m->lset[lev + 1];
    CK(m, timed(m, CC_K_REFINE, [&] { return launch_iface(S, pr, rO, rC, rN, rF, first, st); }), "flux register");
    nl++;
  }
  if (L.ncols > 0) {
    CK(m, timed(m, CC_K_DIAGNOSE, [&] { return launch_diagnose(L, pr, rN, rC, rO, rF, first, 1, st); }),
       "velocity diagnosis");
    nl++;
  }
  int lo = lev < 0 ? 0 : m->lev_first[lev], hi = lev < 0 ? m->ndom : lo + m->lev_count[lev];
  for (int q = lo; q < hi; q++) {
    DomHost &H = m->dom[q];
    int o = H.r[0], c = H.r[1];
    H.r[0] = H.r[3];
    H.r[1] = H.r[2];
    H.r[2] = o;
    H.r[3] = c;
    H.nsteps++;
  }
  // the blocks' ghost shells where they lie in siblings: the new current and
  // the filtered old level, the two the next step reads
  if (lev >= 0 && m->nxch[lev] > 0) {
    CK(m, timed(m, CC_K_REFINE, [&] {
         return launch_exchange(m->d_doms, m->d_xch[lev], m->nxch[lev], pr, H0.r[0], H0.r[1], st);
       }),
       "same-level copies");
    nl++;
  }
  return CC_OK;
}

// cycle(l) of a refined model (Sec 2.2): two steps of level l+1 (each after
// adding the fine fluxes of its current state, the state that step uses, to
// the register), the step of level l with the register, then the register
// is cleared, level l+1 restricted onto level l and level l prolonged into the
// ghost frame of level l+1.
static cc_status cycle(cc_model *m, int l, long long &nl) {
  const int pr = m->prec;
  cudaStream_t st = m->st;
  const bool fine = l + 1 < m->nlev;
  if (fine) {
    const LinkSet &S = m->lset[l + 1];
    const int f0 = m->lev_first[l + 1];
    for (int s = 0; s < 2; s++) {
      CK(m, timed(m, CC_K_REFINE, [&] { return launch_register_add(S, pr, m->dom[f0].r[1], st); }),
         "register add");
      nl++;
      cc_status r = cycle(m, l + 1, nl);
      if (r != CC_OK) return r;
    }
  }
  cc_status r = step_domains(m, l, nl);
  if (r != CC_OK) return r;
  if (fine) {
    // every block restricted before any is prolonged: the injection into a
    // block's shell reads coarse corners that a neighbouring block restricts
    const LinkSet &S = m->lset[l + 1];
    const int f0 = m->lev_first[l + 1], dc = m->lev_first[l];
    CK(m, timed(m, CC_K_REFINE, [&] { return launch_register_clear(S, pr, st); }), "register clear");
    CK(m, timed(m, CC_K_REFINE, [&] { return launch_restrict(S, pr, m->dom[f0].r[1], st); }), "restrict");
    CK(m, timed(m, CC_K_REFINE, [&] { return launch_prolong(S, pr, m->dom[dc].r[1], st); }), "prolong");
    nl += 3;
  }
  return CC_OK;
}

extern "C" {

static cc_status one_step(cc_model *m, long long &nl) { return m->refined ? cycle(m, 0, nl) : step_domains(m, -1, nl); }

static std::vector<int> graph_key(const cc_model *m) {
  std::vector<int> k;
  k.push_back(m->sched);
  k.push_back(m->roles);
  for (const auto &H : m->dom) {
    for (int a = 0; a < 4; a++) k.push_back(H.r[a]);
    k.push_back(H.sched);
    k.push_back(H.roles);
  }
  return k;
}

// One step through a CUDA graph: the launches of the step are captured once
// per key on the private stream and replayed on the model's stream; a replay
// advances the host bookkeeping without launching.
static cc_status graph_step(cc_model *m, long long &nl) {
  const std::vector<int> key = graph_key(m);
  for (auto &g : m->graphs)
    if (g.key == key) {
      m->dry = true;
      long long dummy = 0;
      cc_status r = one_step(m, dummy);
      m->dry = false;
      if (r != CC_OK) return r;
      CK(m, cudaGraphLaunch(g.exec, m->st), "graph launch");
      nl += g.launches;
      return CC_OK;
    }
  if (!m->cap) CK(m, cudaStreamCreateWithFlags(&m->cap, cudaStreamNonBlocking), "capture stream");
  // the capture stream starts after the work already queued on the model's stream
  std::vector<std::array<int, 4>> roles;
  std::vector<long long> steps;
  for (const auto &H : m->dom) {
    roles.push_back({H.r[0], H.r[1], H.r[2], H.r[3]});
    steps.push_back(H.nsteps);
  }
  auto restore = [&]() {
    for (size_t d = 0; d < m->dom.size(); d++) {
      for (int a = 0; a < 4; a++) m->dom[d].r[a] = roles[d][a];
      m->dom[d].nsteps = steps[d];
    }
  };
  cudaStream_t saved = m->st;
  CK(m, cudaStreamBeginCapture(m->cap, cudaStreamCaptureModeThreadLocal), "begin capture");
  m->st = m->cap;
  long long cl = 0;
  cc_status r = one_step(m, cl);
  m->st = saved;
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(m->cap, &graph);
  if (r != CC_OK || e != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    restore();
    return r != CC_OK ? r : cuda_fail(m, e, "end capture");
  }
  cudaGraphExec_t exec = nullptr;
  e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    restore();
    return cuda_fail(m, e, "graph instantiate");
  }
  m->graphs.push_back({key, exec, cl});
  CK(m, cudaGraphLaunch(exec, m->st), "graph launch");
  nl += cl;
  return CC_OK;
}

cc_status cc_step(cc_model *m, int n) {
  if (!m) return fail(m, CC_EINVAL, "null model");
  if (n < 0) return fail(m, CC_EINVAL, "negative step count");
  if (!m->state) return fail(m, CC_ESTATE, "state not initialised");
  // the flags of the earlier calls, if their copy has arrived (no wait)
  if (m->watch_pending && cudaEventQuery(m->ev_watch) == cudaSuccess) {
    cc_status w = watch_verdict(m);
    if (w != CC_OK) return w;
  }
  long long nl = 0;
  cc_status r = CC_OK;
  for (int s = 0; s < n && r == CC_OK; s++) {
    // forward-Euler starts and profiled steps run eagerly
    bool graph = m->graphs_on && !m->prof;
    for (const auto &H : m->dom) graph = graph && H.nsteps > 0;
    r = graph ? graph_step(m, nl) : one_step(m, nl);
  }
  m->last_launches = nl;
  if (r == CC_OK && n > 0) {
    CK(m, cudaMemcpyAsync(m->h_watch, m->d_watch, sizeof(unsigned), cudaMemcpyDeviceToHost, m->st), "watchdog copy");
    CK(m, cudaEventRecord(m->ev_watch, m->st), "watchdog event");
    m->watch_pending = true;
  }
  return r;
}

cc_status cc_inject_wait_timeout(cc_model *m, int on) {
  if (!m) return fail(m, CC_EINVAL, "null model");
  m->stall_tx = on ? 16u : 0u;
  // captured graphs hold the old launch parameters
  CK(m, cudaStreamSynchronize(m->st), "inject sync");
  for (auto &g : m->graphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  m->graphs.clear();
  return CC_OK;
}

cc_status cc_graphs_enable(cc_model *m, int on) {
  if (!m) return fail(m, CC_EINVAL, "null model");
  m->graphs_on = on != 0;
  return CC_OK;
}

// Checkpoint file: a header (magic, version, precision, domain count and
// sizes, time-level roles and step counts) followed, per domain, by the raw
// device arrays of all four time levels (five fields and the boundary-point
// velocity, padded layout, model precision).
namespace {
const char kMagic[8] = {'C', 'U', 'T', 'C', 'E', 'L', 'L', '1'};
constexpr int32_t kCkptVersion = 2;
struct CkptDom {
  int32_t nx, ny, nz, px, py, pz, r[4];
  int64_t nsteps;
  uint64_t fingerprint;  // the domain's configuration and terrain
};

// 64-bit FNV-1a over the domain's configuration (field by field, so that no
// padding byte enters) and its corner heights: a checkpoint written for
// another hill, spacing, time step or flow does not load.
uint64_t fingerprint(const DomHost &H) {
  uint64_t h = 1469598103934665603ull;
  auto mix = [&](const void *p, size_t n) {
    const unsigned char *b = (const unsigned char *)p;
    for (size_t a = 0; a < n; a++) {
      h ^= b[a];
      h *= 1099511628211ull;
    }
  };
  const cc_config &c = H.cfg;
  const int ints[4] = {c.nx, c.ny, c.nz, c.bc_slip};
  const double dbl[16] = {c.dx, c.dy, c.dz, c.dt, c.U, c.N, c.theta0, c.p_surf,
                          c.p0, c.g,  c.R,  c.cp, c.ra_nu, c.c4, c.sponge_frac, c.tau_max};
  mix(ints, sizeof(ints));
  mix(dbl, sizeof(dbl));
  if (!H.hh.empty()) mix(H.hh.data(), H.hh.size() * sizeof(double));
  return h;
}
}  // namespace

cc_status cc_save(const cc_model *mc, const char *path) {
  cc_model *m = const_cast<cc_model *>(mc);
  if (!m || !path) return fail(m, CC_EINVAL, "null argument");
  if (!m->state) return fail(m, CC_ESTATE, "state not initialised");
  CK(m, cudaStreamSynchronize(m->st), "save sync");
  FILE *f = std::fopen(path, "wb");
  if (!f) return fail(m, CC_EINVAL, std::string("cannot open ") + path + " for writing");
  bool ok = std::fwrite(kMagic, 1, 8, f) == 8;
  int32_t hdr[4] = {kCkptVersion, m->prec, m->ndom, m->refined ? 1 : 0};
  ok = ok && std::fwrite(hdr, sizeof(hdr), 1, f) == 1;
  for (const auto &H : m->dom) {
    CkptDom c{H.D.nx, H.D.ny, H.D.nz, H.D.px, H.D.py, H.D.pz, {H.r[0], H.r[1], H.r[2], H.r[3]}, H.nsteps,
              fingerprint(H)};
    ok = ok && std::fwrite(&c, sizeof(c), 1, f) == 1;
  }
  std::vector<char> buf;
  for (const auto &H : m->dom) {
    const size_t nf = (size_t)H.D.ncellp * m->esz, nu = (size_t)3 * H.D.plane * m->esz;
    buf.resize(std::max(nf, nu));
    for (int b = 0; b < NBUF && ok; b++) {
      for (int fl = 0; fl < NFIELD && ok; fl++) {
        cudaError_t e = cudaMemcpy(buf.data(), H.D.f[b][fl], nf, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) {
          std::fclose(f);
          return cuda_fail(m, e, "save copy");
        }
        ok = std::fwrite(buf.data(), 1, nf, f) == nf;
      }
      if (!ok) break;
      cudaError_t e = cudaMemcpy(buf.data(), H.D.ub[b], nu, cudaMemcpyDeviceToHost);
      if (e != cudaSuccess) {
        std::fclose(f);
        return cuda_fail(m, e, "save copy");
      }
      ok = std::fwrite(buf.data(), 1, nu, f) == nu;
    }
  }
  ok = (std::fclose(f) == 0) && ok;
  if (!ok) return fail(m, CC_EINVAL, std::string("write to ") + path + " failed");
  return CC_OK;
}

cc_status cc_load(cc_model *m, const char *path) {
  if (!m || !path) return fail(m, CC_EINVAL, "null argument");
  if (!m->geom) return fail(m, CC_ESTATE, "geometry not built");
  FILE *f = std::fopen(path, "rb");
  if (!f) return fail(m, CC_EINVAL, std::string("cannot open ") + path);
  auto bad = [&](const std::string &why) {
    std::fclose(f);
    return fail(m, CC_EINVAL, std::string(path) + ": " + why);
  };
  char magic[8];
  int32_t hdr[4];
  if (std::fread(magic, 1, 8, f) != 8 || std::memcmp(magic, kMagic, 8) != 0) return bad("not a checkpoint file");
  if (std::fread(hdr, sizeof(hdr), 1, f) != 1 || hdr[0] != kCkptVersion) return bad("unknown checkpoint version");
  if (hdr[1] != m->prec || hdr[2] != m->ndom || hdr[3] != (m->refined ? 1 : 0))
    return bad("precision, domain count or refinement differ from the model");
  std::vector<CkptDom> cd(m->ndom);
  for (int d = 0; d < m->ndom; d++) {
    if (std::fread(&cd[d], sizeof(CkptDom), 1, f) != 1) return bad("truncated header");
    const DomDev &D = m->dom[d].D;
    if (cd[d].nx != D.nx || cd[d].ny != D.ny || cd[d].nz != D.nz || cd[d].px != D.px || cd[d].py != D.py ||
        cd[d].pz != D.pz)
      return bad("domain " + std::to_string(d) + " has other sizes than the model's");
    int seen = 0;
    for (int a = 0; a < 4; a++) {
      if (cd[d].r[a] < 0 || cd[d].r[a] >= NBUF) return bad("invalid time-level roles");
      seen |= 1 << cd[d].r[a];
    }
    if (seen != (1 << NBUF) - 1) return bad("time-level roles of domain " + std::to_string(d) + " repeat a buffer");
    if (cd[d].fingerprint != fingerprint(m->dom[d]))
      return bad("domain " + std::to_string(d) + " was written for another configuration or terrain");
  }
  std::vector<char> buf;
  m->state = false;  // until every array has been read
  for (int d = 0; d < m->ndom; d++) {
    const DomDev &D = m->dom[d].D;
    const size_t nf = (size_t)D.ncellp * m->esz, nu = (size_t)3 * D.plane * m->esz;
    buf.resize(std::max(nf, nu));
    for (int b = 0; b < NBUF; b++) {
      for (int fl = 0; fl < NFIELD; fl++) {
        if (std::fread(buf.data(), 1, nf, f) != nf) return bad("truncated data");
        cudaError_t e = cudaMemcpy(D.f[b][fl], buf.data(), nf, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
          std::fclose(f);
          return cuda_fail(m, e, "load copy");
        }
      }
      if (std::fread(buf.data(), 1, nu, f) != nu) return bad("truncated data");
      cudaError_t e = cudaMemcpy(D.ub[b], buf.data(), nu, cudaMemcpyHostToDevice);
      if (e != cudaSuccess) {
        std::fclose(f);
        return cuda_fail(m, e, "load copy");
      }
    }
  }
  std::fclose(f);
  for (int d = 0; d < m->ndom; d++) {
    for (int a = 0; a < 4; a++) m->dom[d].r[a] = cd[d].r[a];
    m->dom[d].nsteps = cd[d].nsteps;
  }
  // the flux registers are empty between steps
  for (int d = 0; d < (int)m->link.size(); d++) {
    if (m->dom_level[d] == 0) continue;
    const LevelLink &K = m->link[d].L;
    CK(m, cudaMemsetAsync(K.regm, 0, K.nfaces * m->esz, m->st), "register reset");
    CK(m, cudaMemsetAsync(K.regh, 0, K.nfaces * m->esz, m->st), "register reset");
  }
  cc_status w = watch_reset(m);
  if (w != CC_OK) return w;
  CK(m, cudaStreamSynchronize(m->st), "load sync");
  m->state = true;
  return CC_OK;
}

cc_status cc_diagnostics(cc_model *m, int d, cc_diag *out) {
  if (!m || !out) return fail(m, CC_EINVAL, "null argument");
  if (d < 0 || d >= m->ndom) return fail(m, CC_EINVAL, "domain index out of range");
  if (!m->state) return fail(m, CC_ESTATE, "state not initialised");
  const DomHost &H = m->dom[d];
  CK(m, launch_diag_reduce(H.D, m->d_doms + d, m->prec, H.r[1], m->d_diag, m->st), "diagnostics");
  CK(m, launch_heat(m->d_doms + d, m->prec, H.r[1], m->d_diag + 5, m->d_diag + 8 + 5 * 256, m->st), "heat");
  double h[8];
  CK(m, cudaMemcpyAsync(h, m->d_diag, sizeof(double) * 7, cudaMemcpyDeviceToHost, m->st), "diag copy");
  CK(m, cudaStreamSynchronize(m->st), "diag sync");
  out->mass = h[0];
  out->mass_comp = h[1];
  out->max_u = h[2];
  out->max_w = h[3];
  out->nonfinite = (long long)h[4];
  out->steps = H.nsteps;
  out->heat = h[5];
  out->heat_comp = h[6];
  if (out->nonfinite > 0) return fail(m, CC_ENUMERIC, "non-finite values in the state");
  return CC_OK;
}

cc_status cc_refine_mass(cc_model *m, int both, double *out) {
  if (!m || !out) return fail(m, CC_EINVAL, "null argument");
  if (!m->refined) return fail(m, CC_EINVAL, "not a refined model");
  if (!m->state) return fail(m, CC_ESTATE, "state not initialised");
  double tot = 0.0;
  for (int d = 0; d < m->ndom; d++) {
    const DomHost &H = m->dom[d];
    const int l = m->dom_level[d];
    int x0 = 0, x1 = 0, y0 = 0, y1 = 0, z1 = 0;
    if (l + 1 < m->nlev) {
      // the whole box of the next finer level (all its blocks)
      const cc_box &U = m->lev_box[l + 1];
      x0 = U.ox / 2; x1 = (U.ox + U.nx) / 2; y0 = U.oy / 2; y1 = (U.oy + U.ny) / 2; z1 = U.nz / 2;
    }
    CK(m, launch_mass_active(H.D, m->d_doms + d, m->prec, H.r[1], H.r[0], both, x0, x1, y0, y1, z1, m->d_diag,
                             m->st),
       "mass");
    double h = 0.0;
    CK(m, cudaMemcpyAsync(&h, m->d_diag, sizeof(double), cudaMemcpyDeviceToHost, m->st), "mass copy");
    CK(m, cudaStreamSynchronize(m->st), "mass sync");
    tot += h;
  }
  *out = tot;
  return CC_OK;
}

cc_status cc_autotune(cc_model *m, int reps) {
  if (!m) return fail(m, CC_EINVAL, "null model");
  if (reps < 1 || reps > 100) return fail(m, CC_EINVAL, "reps must be 1 .. 100");
  if (!m->state) return fail(m, CC_ESTATE, "state not initialised");
  cudaEvent_t a = nullptr, b = nullptr;
  CK(m, cudaEventCreate(&a), "event");
  if (cudaEventCreate(&b) != cudaSuccess) {
    cudaEventDestroy(a);
    return fail(m, CC_ECUDA, "event");
  }
  cc_status res = CC_OK;
  // launch groups: the whole ensemble, or each level of a refined model (all
  // its blocks, which share the schedule)
  const int ngroup = m->refined ? m->nlev : 1;
  for (int g = 0; g < ngroup && res == CC_OK; g++) {
    const int d = m->refined ? g : -1;
    DomHost &H = m->dom[m->refined ? m->lev_first[g] : 0];
    auto set_sched = [&](int sc, int nr) {
      if (!m->refined) {
        m->sched = sc;
        m->roles = nr;
        return;
      }
      for (int q = m->lev_first[g]; q < m->lev_first[g] + m->lev_count[g]; q++) {
        m->dom[q].sched = sc;
        m->dom[q].roles = nr;
      }
    };
    const int first = H.nsteps == 0;
    const int rO = first ? H.r[1] : H.r[0], rC = H.r[1], rN = H.r[2], rF = H.r[3];
    int best = 0;
    float best_ms = 0;
    // every schedule, and in FP32 with one and with two warp roles
    const int nrmax = m->prec == CC_FP32 ? 2 : 1;
    for (int sr = 0; sr < NSCHED * nrmax && res == CC_OK; sr++) {
      const int sc = sr % NSCHED, nr = 1 + sr / NSCHED;
      set_sched(sc, nr);
      StepLaunch L = make_launch(m, d);
      // the stencil writes only the new and filtered levels, which the next
      // step overwrites with the same values: timing it leaves the state alone
      cudaError_t e = launch_full(L, m->prec, rO, rC, rN, rF, first, m->st);
      if (e == cudaSuccess) e = cudaEventRecord(a, m->st);
      for (int r = 0; r < reps && e == cudaSuccess; r++) e = launch_full(L, m->prec, rO, rC, rN, rF, first, m->st);
      if (e == cudaSuccess) e = cudaEventRecord(b, m->st);
      if (e == cudaSuccess) e = cudaEventSynchronize(b);
      float ms = 0;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
      if (e != cudaSuccess) {
        res = cuda_fail(m, e, "autotune");
        break;
      }
      if (sr == 0 || ms < best_ms) {
        best = sr;
        best_ms = ms;
      }
    }
    set_sched(best % NSCHED, 1 + best / NSCHED);
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (res == CC_OK) m->tuned = true;
  return res;
}

cc_status cc_get_schedule(const cc_model *mc, int d, int *tile_y, int *items_per_launch) {
  cc_model *m = const_cast<cc_model *>(mc);
  if (!m || !tile_y || !items_per_launch) return fail(m, CC_EINVAL, "null argument");
  if (d < 0 || d >= m->ndom) return fail(m, CC_EINVAL, "domain index out of range");
  const int sc = m->refined ? m->dom[d].sched : m->sched;
  *tile_y = sched_tile_y(m->prec, sc);
  *items_per_launch = SCHED_ITEMS[sc];
  return CC_OK;
}

cc_status cc_set_schedule(cc_model *m, int d, int tile_y, int items_per_launch) {
  if (!m) return fail(m, CC_EINVAL, "null model");
  if (d < 0 || d >= m->ndom) return fail(m, CC_EINVAL, "domain index out of range");
  for (int sc = 0; sc < NSCHED; sc++)
    if (sched_tile_y(m->prec, sc) == tile_y && SCHED_ITEMS[sc] == items_per_launch) {
      if (m->refined) {
        // every block of the domain's level (one launch)
        const int l = m->dom_level[d];
        for (int q = m->lev_first[l]; q < m->lev_first[l] + m->lev_count[l]; q++) m->dom[q].sched = sc;
      } else {
        m->sched = sc;
      }
      return CC_OK;
    }
  return fail(m, CC_EINVAL, "no such schedule");
}

cc_status cc_get_warp_roles(const cc_model *mc, int d, int *roles) {
  cc_model *m = const_cast<cc_model *>(mc);
  if (!m || !roles) return fail(m, CC_EINVAL, "null argument");
  if (d < 0 || d >= m->ndom) return fail(m, CC_EINVAL, "domain index out of range");
  *roles = m->refined ? m->dom[d].roles : m->roles;
  return CC_OK;
}

cc_status cc_set_warp_roles(cc_model *m, int d, int roles) {
  if (!m) return fail(m, CC_EINVAL, "null model");
  if (d < 0 || d >= m->ndom) return fail(m, CC_EINVAL, "domain index out of range");
  if (roles != 1 && (roles != 2 || m->prec != CC_FP32))
    return fail(m, CC_EINVAL, "warp roles must be 1, or 2 in FP32");
  if (m->refined) {
    const int l = m->dom_level[d];
    for (int q = m->lev_first[l]; q < m->lev_first[l] + m->lev_count[l]; q++) m->dom[q].roles = roles;
  } else {
    m->roles = roles;
  }
  return CC_OK;
}

cc_status cc_synchronize(cc_model *m) {
  if (!m) return fail(m, CC_EINVAL, "null model");
  CK(m, cudaStreamSynchronize(m->st), "synchronize");
  if (m->watch_pending) return watch_verdict(m);
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
  if (kernel < 0 || kernel > CC_K_REFINE) return fail(m, CC_EINVAL, "bad kernel id");
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
