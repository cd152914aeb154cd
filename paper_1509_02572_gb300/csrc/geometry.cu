// Cut-cell geometry on the GPU in FP64 (paper Sec 2.3 and the stencil set-up
// of Sec 2.4).  Compiled with -fmad=false so that every product and sum is
// rounded exactly as written: the cell classes, merge targets, groups and
// stencil indices are then bit-identical to a CPU evaluation of the same
// formulas, and no near-tie can flip a merge decision between the two.
#include <cuda_runtime.h>
#include <math.h>

#include "cc_internal.h"

namespace cc {
namespace {

constexpr int TPB = 256;

inline unsigned nblk(long long n) { return (unsigned)((n + TPB - 1) / TPB); }

// Gauss-Legendre 8-point rule on [-1,1]: nodes and weights of the standard
// tables (symmetric pairs).
__constant__ double kGLx[4] = {0.1834346424956498049394761, 0.5255324099163289858177390,
                               0.7966664774136267395915539, 0.9602898564975362316835609};
__constant__ double kGLw[4] = {0.3626837833783619829651504, 0.3137066458778872873379622,
                               0.2223810344533744705443560, 0.1012285362903762591525314};

__device__ inline double hcorner(const DomDev &D, int I, int J) {
  return D.h[(long long)wrapi(J, D.ny) * D.nx + wrapi(I, D.nx)];
}

// integral over [0,len] of max(z - h(s), 0) for h linear from ha to hb
__device__ inline double line_int(double z, double ha, double hb, double len) {
  double lo = ha < hb ? ha : hb, hi = ha < hb ? hb : ha;
  if (z >= hi) return len * (z - 0.5 * (ha + hb));
  if (z <= lo) return 0.0;
  double d = z - lo;
  return len * d * d / (2.0 * (hi - lo));
}

// fraction of [0,len] where the linear h lies strictly below z
__device__ inline double line_frac(double z, double ha, double hb) {
  double lo = ha < hb ? ha : hb, hi = ha < hb ? hb : ha;
  if (lo == hi) return z > lo ? 1.0 : 0.0;
  if (z >= hi) return 1.0;
  if (z <= lo) return 0.0;
  return (z - lo) / (hi - lo);
}

__device__ inline double col_f(double s, double z, double h00, double h10, double h01, double h11,
                               double dy, int kind) {
  double ha = h00 + (h10 - h00) * s;
  double hb = h01 + (h11 - h01) * s;
  if (kind == 0) return line_int(z, ha, hb, dy);
  return line_frac(z, ha, hb) * dy;
}

// kind 0: integral over the column footprint of max(z - h, 0); kind 1: area
// of the footprint where h < z.  Integrated along x over the segments between
// the points where the clipping case changes.
__device__ double col_int(double z, double h00, double h10, double h01, double h11, double dx,
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
  for (int a = 1; a < nb; a++) {
    double v = bp[a];
    int b = a - 1;
    while (b >= 0 && bp[b] > v) {
      bp[b + 1] = bp[b];
      b--;
    }
    bp[b + 1] = v;
  }
  double tot = 0.0;
  for (int a = 0; a + 1 < nb; a++) {
    if (bp[a + 1] > bp[a]) {
      double lo = bp[a], hi = bp[a + 1];
      double mid = 0.5 * (lo + hi), half = 0.5 * (hi - lo), s = 0.0;
      for (int q = 0; q < 4; q++) {
        s += kGLw[q] * (col_f(mid - half * kGLx[q], z, h00, h10, h01, h11, dy, kind) +
                        col_f(mid + half * kGLx[q], z, h00, h10, h01, h11, dy, kind));
      }
      tot += s * half;
    }
  }
  return tot * dx;
}

// ---------------------------------------------------------------- columns
__global__ void k_columns(DomDev D, double *hc, double *gx, double *gy, int32_t *kug) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)D.nx * D.ny) return;
  int i = (int)(t % D.nx), j = (int)(t / D.nx);
  double h00 = hcorner(D, i, j), h10 = hcorner(D, i + 1, j), h01 = hcorner(D, i, j + 1),
         h11 = hcorner(D, i + 1, j + 1);
  hc[t] = 0.25 * (h00 + h10 + h01 + h11);
  // column gradients, Eqs. xgrad / ygrad
  gx[t] = ((h10 + h11) - (h00 + h01)) / (2.0 * D.dx);
  gy[t] = ((h01 + h11) - (h00 + h10)) / (2.0 * D.dy);
  double hmin = fmin(fmin(h00, h10), fmin(h01, h11));
  int k = 0;
  while (k < D.nz && (k + 1) * D.dz <= hmin) k++;
  kug[qidx(D, i, j)] = k;
}

// ---------------------------------------------------------------- cells
__global__ void k_cells(DomDev D, const double *hc, double *vf, int8_t *cls) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long n = (long long)D.nx * D.ny * D.nz;
  if (t >= n) return;
  int i = (int)(t % D.nx), j = (int)((t / D.nx) % D.ny), k = (int)(t / ((long long)D.nx * D.ny));
  double h00 = hcorner(D, i, j), h10 = hcorner(D, i + 1, j), h01 = hcorner(D, i, j + 1),
         h11 = hcorner(D, i + 1, j + 1);
  double hmin = fmin(fmin(h00, h10), fmin(h01, h11));
  double hmax = fmax(fmax(h00, h10), fmax(h01, h11));
  double z0 = k * D.dz, z1 = (k + 1) * D.dz;
  if (z1 <= hmin) {
    vf[t] = 0.0;
    cls[t] = C_UG;
    return;
  }
  if (z0 >= hmax) {
    vf[t] = 1.0;
    cls[t] = C_FULL;
    return;
  }
  double w1 = col_int(z1, h00, h10, h01, h11, D.dx, D.dy, 0);
  double w0 = col_int(z0, h00, h10, h01, h11, D.dx, D.dy, 0);
  double v = (w1 - w0) / (D.dx * D.dy * D.dz);
  vf[t] = v;
  // merge criterion (Sec 2.3): centre below the terrain or volume below half
  double zc = (k + 0.5) * D.dz;
  bool small = (hc[(long long)j * D.nx + i] > zc) || (v < 0.5);
  cls[t] = small ? C_ABS : C_CUT;
}

// lateral apertures (closed form along each vertical face) and horizontal
// apertures; the floor and the lid are walls
__global__ void k_faces(DomDev D, double *ax, double *ay) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long n = (long long)D.nx * D.ny * D.nz;
  if (t >= n) return;
  int I = (int)(t % D.nx), j = (int)((t / D.nx) % D.ny), k = (int)(t / ((long long)D.nx * D.ny));
  double z0 = k * D.dz, z1 = (k + 1) * D.dz;
  double ha = hcorner(D, I, j), hb = hcorner(D, I, j + 1);
  double a;
  if (z0 >= fmax(ha, hb)) a = 1.0;
  else if (z1 <= fmin(ha, hb)) a = 0.0;
  else a = (line_int(z1, ha, hb, D.dy) - line_int(z0, ha, hb, D.dy)) / (D.dy * D.dz);
  ax[t] = a;
  double ya = hcorner(D, I, j), yb = hcorner(D, I + 1, j);
  if (z0 >= fmax(ya, yb)) a = 1.0;
  else if (z1 <= fmin(ya, yb)) a = 0.0;
  else a = (line_int(z1, ya, yb, D.dx) - line_int(z0, ya, yb, D.dx)) / (D.dx * D.dz);
  ay[t] = a;
}

__global__ void k_zfaces(DomDev D, double *az) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long n = (long long)D.nx * D.ny * (D.nz + 1);
  if (t >= n) return;
  int i = (int)(t % D.nx), j = (int)((t / D.nx) % D.ny), K = (int)(t / ((long long)D.nx * D.ny));
  double a = 0.0;
  if (K > 0 && (K < D.nz || !D.lid)) {
    double z = K * D.dz;
    double h00 = hcorner(D, i, j), h10 = hcorner(D, i + 1, j), h01 = hcorner(D, i, j + 1),
           h11 = hcorner(D, i + 1, j + 1);
    double hmin = fmin(fmin(h00, h10), fmin(h01, h11));
    double hmax = fmax(fmax(h00, h10), fmax(h01, h11));
    if (z > hmax) a = 1.0;
    else if (z <= hmin) a = 0.0;
    else a = col_int(z, h00, h10, h01, h11, D.dx, D.dy, 1) / (D.dx * D.dy);
  }
  az[t] = a;
}

// merge direction of the Fig. 6 pseudocode
__global__ void k_targets(DomDev D, const double *gx, const double *gy, const int8_t *cls,
                          int32_t *target, int *err) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long n = (long long)D.nx * D.ny * D.nz;
  if (t >= n) return;
  target[t] = -1;
  if (cls[t] != C_ABS) return;
  int i = (int)(t % D.nx), j = (int)((t / D.nx) % D.ny), k = (int)(t / ((long long)D.nx * D.ny));
  double g1 = gx[(long long)j * D.nx + i], g2 = gy[(long long)j * D.nx + i];
  double a1 = fabs(g1), a2 = fabs(g2);
  int ti = i, tj = j, tk = k;
  if (a1 <= 1.0 && a2 <= 1.0) {
    tk = k + 1;
    if (tk >= D.nz) {
      atomicOr(err, 1);
      return;
    }
  } else if (g1 > 1.0 && a1 >= a2) {
    ti = i - 1;
  } else if (g1 < -1.0 && a1 >= a2) {
    ti = i + 1;
  } else if (g2 > 1.0 && a1 < a2) {
    tj = j - 1;
  } else {
    tj = j + 1;
  }
  target[t] = (int32_t)(((long long)tk * D.ny + wrapi(tj, D.ny)) * D.nx + wrapi(ti, D.nx));
}

__global__ void k_roots(DomDev D, const int8_t *cls, const int32_t *target, int32_t *root,
                        int8_t *mark, int *err) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long n = (long long)D.nx * D.ny * D.nz;
  if (t >= n) return;
  if (cls[t] == C_UG) {
    root[t] = -1;
    return;
  }
  long long r = t;
  int steps = 0;
  while (cls[r] == C_ABS) {
    r = target[r];
    if (r < 0 || ++steps > 64) {
      atomicOr(err, 2);
      root[t] = -1;
      return;
    }
  }
  if (cls[r] == C_UG) {
    atomicOr(err, 2);
    root[t] = -1;
    return;
  }
  root[t] = (int32_t)r;
  if (cls[t] == C_ABS) mark[r] = 1;  // the host has at least one absorbed member
}

// ---------------------------------------------------------------- compaction
// Stable compaction of indices whose flag is set: per-block counts, one scan
// of the block counts, then a block-local scan and scatter.
__global__ void k_flag_count(const int8_t *flag, long long n, int *bcount) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  int f = (t < n) ? (flag[t] != 0) : 0;
  int c = __syncthreads_count(f);
  if (threadIdx.x == 0) bcount[blockIdx.x] = c;
}

// exclusive scan of n ints by one block; total in out[n]
__global__ void k_scan_single(const int *in, int *out, int n) {
  __shared__ int warp_sums[32];
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < n; base += blockDim.x) {
    int idx = base + threadIdx.x;
    int v = idx < n ? in[idx] : 0;
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int x = v;
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[w] = x;
    __syncthreads();
    if (w == 0) {
      int nw = blockDim.x >> 5;
      int s = lane < nw ? warp_sums[lane] : 0;
      for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, s, o);
        if (lane >= o) s += y;
      }
      if (lane < nw) warp_sums[lane] = s;
    }
    __syncthreads();
    int excl = x - v + (w > 0 ? warp_sums[w - 1] : 0) + carry;
    if (idx < n) out[idx] = excl;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry = excl + v;
    __syncthreads();
  }
  if (threadIdx.x == 0) out[n] = carry;
}

__global__ void k_flag_scatter(const int8_t *flag, long long n, const int *boff, int32_t *out,
                               int32_t *pos) {
  __shared__ int warp_sums[TPB / 32];
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  int f = (t < n) ? (flag[t] != 0) : 0;
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  unsigned bal = __ballot_sync(0xffffffffu, f);
  int before = __popc(bal & ((1u << lane) - 1u));
  if (lane == 0) warp_sums[w] = __popc(bal);
  __syncthreads();
  int woff = 0;
  for (int a = 0; a < w; a++) woff += warp_sums[a];
  if (f) {
    int p = boff[blockIdx.x] + woff + before;
    out[p] = (int32_t)t;
    if (pos) pos[t] = p;
  }
}

// groups: hosts of cut cells and of merged groups
__global__ void k_group_flags(DomDev D, const int8_t *cls, const int32_t *root, const int8_t *mark,
                              int8_t *flag, int32_t *gindex) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long n = (long long)D.nx * D.ny * D.nz;
  if (t >= n) return;
  gindex[t] = -1;
  int8_t c = cls[t];
  flag[t] = (c != C_UG && root[t] == (int32_t)t && (c == C_CUT || mark[t])) ? 1 : 0;
}

__global__ void k_member_count(DomDev D, const int32_t *root, const int32_t *gindex, int *cnt) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long n = (long long)D.nx * D.ny * D.nz;
  if (t >= n) return;
  int32_t r = root[t];
  if (r < 0) return;
  int g = gindex[r];
  if (g >= 0) atomicAdd(&cnt[g], 1);
}

__global__ void k_member_fill(DomDev D, const int32_t *root, const int32_t *gindex, const int *start,
                              int *fill, int32_t *members) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long n = (long long)D.nx * D.ny * D.nz;
  if (t >= n) return;
  int32_t r = root[t];
  if (r < 0) return;
  int g = gindex[r];
  if (g < 0) return;
  int p = atomicAdd(&fill[g], 1);
  members[start[g] + p] = (int32_t)t;
}

// sort each group's members ascending and sum the group volume in that order
__global__ void k_group_finish(DomDev D, int ng, const int32_t *hosts, const int *start,
                               int32_t *members, GroupRec *recs, int dom) {
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= ng) return;
  int s = start[g], e = start[g + 1];
  for (int a = s + 1; a < e; a++) {
    int32_t v = members[a];
    int b = a - 1;
    while (b >= s && members[b] > v) {
      members[b + 1] = members[b];
      b--;
    }
    members[b + 1] = v;
  }
  double vol = 0.0;
  for (int a = s; a < e; a++) vol += D.vf[members[a]] * D.dx * D.dy * D.dz;
  GroupRec r;
  r.dom = dom;
  r.host = hosts[g];
  r.start = s;
  r.count = e - s;
  r.vg = vol;
  recs[g] = r;
}

// ---------------------------------------------------------------- velocity points
__global__ void k_vcls(DomDev D, const int8_t *cls, const int32_t *root, int8_t *vcls) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long n = (long long)D.nx * D.ny * (D.nz + 2 * GH);
  if (t >= n) return;
  int I = (int)(t % D.nx), J = (int)((t / D.nx) % D.ny), K = (int)(t / ((long long)D.nx * D.ny)) - GH;
  int8_t v;
  if (K * D.dz <= hcorner(D, I, J)) {
    v = V_UG;
  } else if (D.lid && K >= D.nz) {
    v = V_LID;
  } else if (K < 1) {
    v = V_MF;
  } else {
    // cells above the box top of a refined level lie over flat floor: owners
    bool own = true;
    for (int dk = -1; dk <= 0; dk++)
      for (int dj = -1; dj <= 0; dj++)
        for (int di = -1; di <= 0; di++) {
          if (K + dk >= D.nz) continue;
          long long c = (((long long)(K + dk)) * D.ny + wrapi(J + dj, D.ny)) * D.nx + wrapi(I + di, D.nx);
          if (cls[c] == C_UG || root[c] != (int32_t)c) own = false;
        }
    v = own ? V_PRED : V_MF;
  }
  vcls[pidx(D, I, J, K)] = v;
}

__device__ inline int8_t vcls_at(const DomDev &D, const int8_t *vcls, int I, int J, int K) {
  return vcls[pidx(D, wrapi(I, D.nx), wrapi(J, D.ny), K)];
}

// boundary points: unit normal from the corner gradients of the column-centre
// heights; nearest plane of predicted points crossed by the normal line
__global__ void k_bstencil(DomDev D, const double *hc, const int8_t *vcls, int32_t *bK, int32_t *bI,
                           int32_t *bJ, double *ba, double *bb, double *bn, int *err) {
  long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t0 >= (long long)D.nx * D.ny) return;
  int I = (int)(t0 % D.nx), J = (int)(t0 / D.nx);
  const long long t = qidx(D, I, J);
  auto HCc = [&](int i, int j) { return hc[(long long)wrapi(j, D.ny) * D.nx + wrapi(i, D.nx)]; };
  if (D.lid && vcls_at(D, vcls, I, J, D.nz - 1) != V_PRED) atomicOr(err, 4);
  const int ktopsearch = D.lid ? D.nz - 1 : D.nz + 1;
  double hm = HCc(I - 1, J - 1), h0m = HCc(I, J - 1), hm0 = HCc(I - 1, J), h00 = HCc(I, J);
  double gxc = ((h0m + h00) - (hm + hm0)) / (2.0 * D.dx);
  double gyc = ((hm0 + h00) - (hm + h0m)) / (2.0 * D.dy);
  double nrm = sqrt(gxc * gxc + gyc * gyc + 1.0);
  double nxv = -gxc / nrm, nyv = -gyc / nrm, nzv = 1.0 / nrm;
  bn[3 * t] = nxv;
  bn[3 * t + 1] = nyv;
  bn[3 * t + 2] = nzv;
  double hh = hcorner(D, I, J);
  int K0 = 0;
  while (K0 * D.dz <= hh) K0++;
  for (int K = K0; K < K0 + 8 && K <= ktopsearch; K++) {
    double tt = (K * D.dz - hh) / nzv;
    // position from the level's indices (a block's origin offsets them), so
    // that a block and the whole level round alike
    double xN = (I + D.gox) * D.dx + tt * nxv, yN = (J + D.goy) * D.dy + tt * nyv;
    double fi = floor(xN / D.dx), fj = floor(yN / D.dy);
    int i0 = (int)fi - D.gox, j0 = (int)fj - D.goy;
    double a = xN / D.dx - fi, b = yN / D.dy - fj;
    bool ok = vcls_at(D, vcls, i0, j0, K) == V_PRED &&
              (a == 0.0 || vcls_at(D, vcls, i0 + 1, j0, K) == V_PRED) &&
              (b == 0.0 || vcls_at(D, vcls, i0, j0 + 1, K) == V_PRED) &&
              (a == 0.0 || b == 0.0 || vcls_at(D, vcls, i0 + 1, j0 + 1, K) == V_PRED);
    if (ok) {
      bK[t] = K;
      bI[t] = D.periodic ? wrapi(i0, D.nx) : i0;
      bJ[t] = D.periodic ? wrapi(j0, D.ny) : j0;
      ba[t] = a;
      bb[t] = b;
      return;
    }
  }
  bK[t] = -1;
  atomicOr(err, 8);
}

// merged-face points: interpolation between the boundary point and the
// nearest predicted point above on the same vertical line
__global__ void k_mstencil(DomDev D, const int8_t *vcls, int32_t *mK, double *mg, int *err) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long n = (long long)D.nx * D.ny * (D.nz + 2 * GH);
  if (t >= n) return;
  int I = (int)(t % D.nx), J = (int)((t / D.nx) % D.ny), K = (int)(t / ((long long)D.nx * D.ny)) - GH;
  long long p = pidx(D, I, J, K);
  mK[p] = -1;
  mg[p] = 0.0;
  if (vcls[p] != V_MF) return;
  int ka = -1;
  const int ktopsearch = D.lid ? D.nz - 1 : D.nz + 1;
  for (int K2 = K + 1; K2 <= ktopsearch; K2++)
    if (vcls[pidx(D, I, J, K2)] == V_PRED) {
      ka = K2;
      break;
    }
  if (ka < 0) {
    atomicOr(err, 16);
    return;
  }
  double hh = hcorner(D, I, J);
  mK[p] = ka;
  mg[p] = (K * D.dz - hh) / (ka * D.dz - hh);
}

// highest non-predicted corner level below the lid, per column
__global__ void k_ktop(DomDev D, const int8_t *vcls, int32_t *ktop) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)D.nx * D.ny) return;
  int I = (int)(t % D.nx), J = (int)(t / D.nx);
  int kt = -GH;
  const int kend = D.lid ? D.nz : D.ck1;
  for (int K = -GH; K < kend; K++)
    if (vcls[pidx(D, I, J, K)] != V_PRED) kt = K;
  ktop[qidx(D, I, J)] = kt;
}

// Columns of a refined level's padded frame lie over flat floor (h = 0):
// predicted above the floor, boundary point at the floor corner with the
// vertical normal and the corner above as its nearest plane.
__global__ void k_flat_columns(DomDev D) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)D.px * D.py) return;
  int I = (int)(t % D.px) - GX, J = (int)(t / D.px) - GH;
  if (I >= 0 && I < D.nx && J >= 0 && J < D.ny) return;
  const_cast<int32_t *>(D.kug)[t] = 0;
  const_cast<int32_t *>(D.bK)[t] = 1;
  const_cast<int32_t *>(D.bI)[t] = I;
  const_cast<int32_t *>(D.bJ)[t] = J;
  const_cast<double *>(D.ba)[t] = 0.0;
  const_cast<double *>(D.bb)[t] = 0.0;
  double *bn = const_cast<double *>(D.bn);
  bn[3 * t] = 0.0;
  bn[3 * t + 1] = 0.0;
  bn[3 * t + 2] = 1.0;
  const_cast<int32_t *>(D.ktop)[t] = 0;
  int8_t *vcls = const_cast<int8_t *>(D.vcls);
  for (int K = -GH; K < D.nz + GH; K++) vcls[pidx(D, I, J, K)] = K <= 0 ? V_UG : V_PRED;
}

// Highest corner level at or below the terrain per padded column (the test
// K dz <= h of the velocity-point classes); KB_NONE outside the integrated
// corner columns of a refined box.  A box's frame lies over flat floor.
__global__ void k_kb(DomDev D, int32_t *kb) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)D.px * D.py) return;
  int I = (int)(t % D.px) - GX, J = (int)(t / D.px) - GH;
  if (!D.periodic && !(I >= D.qi0 && I < D.ci1 && J >= D.qj0 && J < D.cj1)) {
    kb[t] = KB_NONE;
    return;
  }
  bool inside = I >= 0 && I < D.nx && J >= 0 && J < D.ny;
  double h = (D.periodic || inside) ? hcorner(D, I, J) : 0.0;
  int K = -GH;
  while (K + 1 < D.nz + GH && (K + 1) * D.dz <= h) K++;
  kb[t] = K;
}

// Lowest fluid cell level of column (i, j) (full or cut: the classes of a
// column run below-terrain, absorbed, cut, full upwards) and lowest fluid
// corner level of corner column (I, J) (K dz above the terrain height, K >= 1).
// A refined box's frame lies over flat floor.
__device__ int first_fluid_cell(const DomDev &D, int i, int j) {
  if (D.periodic) {
    i = wrapi(i, D.nx);
    j = wrapi(j, D.ny);
  } else if (i < 0 || i >= D.nx || j < 0 || j >= D.ny) {
    return 0;
  }
  for (int k = 0; k < D.nz; k++) {
    const int8_t c = D.cls[cid(D, i, j, k)];
    if (c == C_FULL || c == C_CUT) return k;
  }
  return D.nz;
}
__device__ int first_fluid_corner(const DomDev &D, int I, int J) {
  const bool inside = I >= 0 && I < D.nx && J >= 0 && J < D.ny;
  const double h = (D.periodic || inside) ? hcorner(D, I, J) : 0.0;
  int K = 1;
  while (K < D.nz + GH && K * D.dz <= h) K++;
  return K;
}

// Reach of the diffusion stencils of every padded column (the descriptor of
// the header): the lowest fluid levels of the column and of its neighbours at
// -2 .. +2 along x and y, the lid, and the band of levels in which the cell
// (x: its neighbours fluid; z: the two cells below fluid, the two above below
// the lid) and the corner (likewise) both take the fourth-order term.
__global__ void k_diffcols(DomDev D, DiffCol *out) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)D.px * D.py) return;
  const int i = (int)(t % D.px) - GX, j = (int)(t / D.px) - GH;
  const int off[4] = {-2, -1, 1, 2};
  DiffCol q;
  const int big = 16000;
  q.ctop = (int16_t)(D.lid ? D.nz : big);
  q.vtop = (int16_t)(D.lid ? D.nz : big);
  int c0 = first_fluid_cell(D, i, j), v0 = first_fluid_corner(D, i, j);
  q.c0 = (int16_t)c0;
  q.v0 = (int16_t)v0;
  int lo = max(c0 + 2, v0 + 2);
  for (int a = 0; a < 4; a++) {
    const int cxa = first_fluid_cell(D, i + off[a], j), cya = first_fluid_cell(D, i, j + off[a]);
    const int vxa = first_fluid_corner(D, i + off[a], j), vya = first_fluid_corner(D, i, j + off[a]);
    q.cx[a] = (int16_t)cxa;
    q.cy[a] = (int16_t)cya;
    q.vx[a] = (int16_t)vxa;
    q.vy[a] = (int16_t)vya;
    lo = max(lo, max(max(cxa, cya), max(vxa, vya)));
  }
  q.lo = (int16_t)lo;
  q.hi = (int16_t)(D.lid ? D.nz - 2 : big);
  out[t] = q;
}

}  // namespace

cudaError_t launch_diffcols(const DomDev &D, cudaStream_t st) {
  k_diffcols<<<nblk((long long)D.px * D.py), TPB, 0, st>>>(D, const_cast<DiffCol *>(D.dcol));
  return cudaGetLastError();
}

// Analytic hill at the corners (I dx, J dy) relative to its centre (xc, yc):
// the bell-shaped hill h0 / (1 + r^2/a^2)^(3/2) (Sec 3.1.1), the half-
// ellipsoid h0 sqrt(1 - r^2/a^2) (the hemisphere of Sec 3.1.2 when h0 = a)
// and the cosine hill h0 (1 + cos(pi r / a)) / 2 for r < a (appendix).  This
// unit is compiled without contraction, so every operation rounds as written.
__global__ void k_hill(double *h, int nx, int ny, double dx, double dy, int kind, double h0, double a, double xc,
                       double yc) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)nx * ny) return;
  const int I = (int)(t % nx), J = (int)(t / nx);
  const double x = (double)I * dx - xc, y = (double)J * dy - yc;
  const double r2 = x * x + y * y;
  double v = 0.0;
  if (kind == CC_HILL_BELL) {
    v = h0 / pow(1.0 + r2 / (a * a), 1.5);
  } else if (kind == CC_HILL_ELLIPSOID) {
    v = h0 * sqrt(fmax(0.0, 1.0 - r2 / (a * a)));
  } else if (kind == CC_HILL_COSINE) {
    const double r = sqrt(r2);
    v = r < a ? 0.5 * h0 * (1.0 + cos(M_PI * r / a)) : 0.0;
  }
  h[t] = v;
}

cudaError_t launch_hill(double *h, int nx, int ny, double dx, double dy, int kind, double h0, double a, double xc,
                        double yc, cudaStream_t st) {
  long long n = (long long)nx * ny;
  k_hill<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(h, nx, ny, dx, dy, kind, h0, a, xc, yc);
  return cudaGetLastError();
}

cudaError_t launch_flat_columns(const DomDev &D, cudaStream_t st) {
  k_flat_columns<<<nblk((long long)D.px * D.py), TPB, 0, st>>>(D);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- driver
struct GeomScratch {
  double *hc = nullptr, *gx = nullptr, *gy = nullptr;
  int32_t *target = nullptr, *gindex = nullptr, *glist = nullptr;
  int8_t *mark = nullptr, *flag = nullptr;
  int *bcount = nullptr, *boff = nullptr, *cnt = nullptr, *start = nullptr, *fill = nullptr;
};

#define GK(call)                           \
  do {                                     \
    cudaError_t e_ = (call);               \
    if (e_ != cudaSuccess) return e_;      \
  } while (0)

// Builds the geometry of one domain.  Writes the geometry arrays whose device
// pointers are in *D (cast away const: the model owns them) and returns the
// group list through the out pointers (device allocations owned by the caller).
cudaError_t geom_build_one(DomDev &D, cudaStream_t st, int dom, int *d_err, int32_t **members_out,
                           GroupRec **recs_out, int *ng_out, int *nm_out) {
  long long ncol = (long long)D.nx * D.ny;
  long long ncell = ncol * D.nz;
  long long ncorner = ncol * (D.nz + 2 * GH);
  GeomScratch S;
  cudaError_t err = cudaSuccess;
  auto cleanup = [&]() {
    cudaFree(S.hc); cudaFree(S.gx); cudaFree(S.gy); cudaFree(S.target); cudaFree(S.gindex);
    cudaFree(S.glist); cudaFree(S.mark); cudaFree(S.flag); cudaFree(S.bcount); cudaFree(S.boff);
    cudaFree(S.cnt); cudaFree(S.start); cudaFree(S.fill);
  };
  do {
    if ((err = cudaMalloc(&S.hc, ncol * 8)) != cudaSuccess) break;
    if ((err = cudaMalloc(&S.gx, ncol * 8)) != cudaSuccess) break;
    if ((err = cudaMalloc(&S.gy, ncol * 8)) != cudaSuccess) break;
    if ((err = cudaMalloc(&S.target, ncell * 4)) != cudaSuccess) break;
    if ((err = cudaMalloc(&S.gindex, ncell * 4)) != cudaSuccess) break;
    if ((err = cudaMalloc(&S.glist, ncell * 4)) != cudaSuccess) break;
    if ((err = cudaMalloc(&S.mark, ncell)) != cudaSuccess) break;
    if ((err = cudaMalloc(&S.flag, ncell)) != cudaSuccess) break;
    unsigned nb = nblk(ncell);
    if ((err = cudaMalloc(&S.bcount, (size_t)(nb + 1) * 4)) != cudaSuccess) break;
    if ((err = cudaMalloc(&S.boff, (size_t)(nb + 1) * 4)) != cudaSuccess) break;
    if ((err = cudaMemsetAsync(S.mark, 0, ncell, st)) != cudaSuccess) break;

    double *vf = const_cast<double *>(D.vf);
    double *ax = const_cast<double *>(D.ax), *ay = const_cast<double *>(D.ay);
    double *az = const_cast<double *>(D.az);
    int8_t *cls = const_cast<int8_t *>(D.cls);
    int32_t *root = const_cast<int32_t *>(D.root);
    int32_t *kug = const_cast<int32_t *>(D.kug);
    int8_t *vcls = const_cast<int8_t *>(D.vcls);
    int32_t *mK = const_cast<int32_t *>(D.mK);
    double *mg = const_cast<double *>(D.mg);

    k_columns<<<nblk(ncol), TPB, 0, st>>>(D, S.hc, S.gx, S.gy, kug);
    k_cells<<<nblk(ncell), TPB, 0, st>>>(D, S.hc, vf, cls);
    k_faces<<<nblk(ncell), TPB, 0, st>>>(D, ax, ay);
    k_zfaces<<<nblk(ncol * (D.nz + 1)), TPB, 0, st>>>(D, az);
    k_targets<<<nblk(ncell), TPB, 0, st>>>(D, S.gx, S.gy, cls, S.target, d_err);
    k_roots<<<nblk(ncell), TPB, 0, st>>>(D, cls, S.target, root, S.mark, d_err);
    k_group_flags<<<nblk(ncell), TPB, 0, st>>>(D, cls, root, S.mark, S.flag, S.gindex);
    k_flag_count<<<nb, TPB, 0, st>>>(S.flag, ncell, S.bcount);
    k_scan_single<<<1, 1024, 0, st>>>(S.bcount, S.boff, (int)nb);
    k_flag_scatter<<<nb, TPB, 0, st>>>(S.flag, ncell, S.boff, S.glist, S.gindex);
    if ((err = cudaGetLastError()) != cudaSuccess) break;
    int ng = 0;
    if ((err = cudaMemcpyAsync(&ng, S.boff + nb, 4, cudaMemcpyDeviceToHost, st)) != cudaSuccess) break;
    if ((err = cudaStreamSynchronize(st)) != cudaSuccess) break;
    if ((err = cudaMalloc(&S.cnt, (size_t)(ng + 1) * 4)) != cudaSuccess) break;
    if ((err = cudaMalloc(&S.start, (size_t)(ng + 1) * 4)) != cudaSuccess) break;
    if ((err = cudaMalloc(&S.fill, (size_t)(ng + 1) * 4)) != cudaSuccess) break;
    if ((err = cudaMemsetAsync(S.cnt, 0, (size_t)(ng + 1) * 4, st)) != cudaSuccess) break;
    if ((err = cudaMemsetAsync(S.fill, 0, (size_t)(ng + 1) * 4, st)) != cudaSuccess) break;
    k_member_count<<<nblk(ncell), TPB, 0, st>>>(D, root, S.gindex, S.cnt);
    k_scan_single<<<1, 1024, 0, st>>>(S.cnt, S.start, ng);
    int nm = 0;
    if ((err = cudaMemcpyAsync(&nm, S.start + ng, 4, cudaMemcpyDeviceToHost, st)) != cudaSuccess) break;
    if ((err = cudaStreamSynchronize(st)) != cudaSuccess) break;
    int32_t *members = nullptr;
    GroupRec *recs = nullptr;
    if ((err = cudaMalloc(&members, (size_t)(nm > 0 ? nm : 1) * 4)) != cudaSuccess) break;
    if ((err = cudaMalloc(&recs, (size_t)(ng > 0 ? ng : 1) * sizeof(GroupRec))) != cudaSuccess) {
      cudaFree(members);
      break;
    }
    k_member_fill<<<nblk(ncell), TPB, 0, st>>>(D, root, S.gindex, S.start, S.fill, members);
    if (ng > 0) k_group_finish<<<nblk(ng), TPB, 0, st>>>(D, ng, S.glist, S.start, members, recs, dom);

    k_vcls<<<nblk(ncorner), TPB, 0, st>>>(D, cls, root, vcls);
    k_bstencil<<<nblk(ncol), TPB, 0, st>>>(D, S.hc, vcls, const_cast<int32_t *>(D.bK),
                                           const_cast<int32_t *>(D.bI), const_cast<int32_t *>(D.bJ),
                                           const_cast<double *>(D.ba), const_cast<double *>(D.bb),
                                           const_cast<double *>(D.bn), d_err);
    k_mstencil<<<nblk(ncorner), TPB, 0, st>>>(D, vcls, mK, mg, d_err);
    k_ktop<<<nblk(ncol), TPB, 0, st>>>(D, vcls, const_cast<int32_t *>(D.ktop));
    k_kb<<<nblk((long long)D.px * D.py), TPB, 0, st>>>(D, const_cast<int32_t *>(D.kb));
    if ((err = cudaGetLastError()) != cudaSuccess) {
      cudaFree(members);
      cudaFree(recs);
      break;
    }
    if ((err = cudaStreamSynchronize(st)) != cudaSuccess) {
      cudaFree(members);
      cudaFree(recs);
      break;
    }
    *members_out = members;
    *recs_out = recs;
    *ng_out = ng;
    *nm_out = nm;
  } while (0);
  cleanup();
  return err;
}

}  // namespace cc
