// Block-structured cube layout (Sec 2.2, the grid generation of the
// cube-based Cartesian mesh): host code.
//
// The domain is divided into equal cubes; cubes near the terrain are split
// into eight, level after level; neighbouring cubes (faces, edges, corners)
// are then made to differ by at most one level; cubes completely inside the
// terrain are dropped. Refinement test (the paper only says that cubes close
// to the terrain surface are split; this test reproduces its cube counts): a
// cube below the finest level is split when its bottom lies below the highest
// terrain point and its footprint lies within one cube width, horizontally,
// of a column where the terrain is raised above its lowest value. Lateral
// boundaries are periodic.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include "cc_internal.h"

namespace {

struct Layout {
  int nlev, L;
  std::vector<int> ncx, ncy, ncz;
  std::vector<std::vector<uint8_t>> refined;  // per level, cube index (ck*ncy + cj)*ncx + ci
  size_t idx(int l, int ci, int cj, int ck) const { return ((size_t)ck * ncy[l] + cj) * ncx[l] + ci; }
  bool is_ref(int l, int ci, int cj, int ck) const { return l < L && refined[l][idx(l, ci, cj, ck)]; }
  bool exists(int l, int ci, int cj, int ck) const { return l == 0 || is_ref(l - 1, ci / 2, cj / 2, ck / 2); }
};

// distance from p to the interval [a0, a1] on a circle of length period
double axis_gap(double p, double a0, double a1, double period) {
  double best = 1e300;
  for (int s = -1; s <= 1; s++) {
    const double q = p + s * period;
    best = std::min(best, std::max(0.0, std::max(a0 - q, q - a1)));
  }
  return best;
}

}  // namespace

extern "C" cc_status cc_cbcm_cubes(int nx0, int ny0, int nz0, int cube, double H, int nlev, const double *h_finest,
                                   cc_cube *out, int capacity, int *count) {
  if (!h_finest || !count || nlev < 1 || nlev > 12 || cube < 1 || nx0 < cube || ny0 < cube || nz0 < cube ||
      nx0 % cube || ny0 % cube || nz0 % cube || !(H > 0))
    return CC_EINVAL;
  Layout T;
  T.nlev = nlev;
  T.L = nlev - 1;
  const int L = T.L;
  const long long fnx = (long long)nx0 << L, fny = (long long)ny0 << L;
  if (fnx * fny > (1LL << 34)) return CC_EINVAL;
  const double Lx = nx0 * H, Ly = ny0 * H, df = H / (double)(1LL << L);
  double hmin = h_finest[0], hmax = h_finest[0];
  for (long long q = 0; q < fnx * fny; q++) {
    if (!std::isfinite(h_finest[q])) return CC_EINVAL;
    hmin = std::min(hmin, h_finest[q]);
    hmax = std::max(hmax, h_finest[q]);
  }
  std::vector<double> rx, ry;  // raised corner points
  for (long long J = 0; J < fny; J++)
    for (long long I = 0; I < fnx; I++)
      if (h_finest[J * fnx + I] > hmin) {
        rx.push_back(I * df);
        ry.push_back(J * df);
      }
  for (int l = 0; l < nlev; l++) {
    T.ncx.push_back((nx0 / cube) << l);
    T.ncy.push_back((ny0 / cube) << l);
    T.ncz.push_back((nz0 / cube) << l);
  }
  long long total = 0;
  for (int l = 0; l < L; l++) {
    const long long n = (long long)T.ncx[l] * T.ncy[l] * T.ncz[l];
    total += n;
    if (total > (1LL << 31)) return CC_EINVAL;
    T.refined.emplace_back((size_t)n, 0);
  }
  auto size = [&](int l) { return cube * H / (double)(1LL << l); };
  // refinement by the terrain test, level by level
  for (int l = 0; l < L; l++) {
    const double s = size(l);
    for (int ck = 0; ck < T.ncz[l]; ck++) {
      if (!(ck * s < hmax)) continue;
      for (int cj = 0; cj < T.ncy[l]; cj++)
        for (int ci = 0; ci < T.ncx[l]; ci++) {
          if (!T.exists(l, ci, cj, ck)) continue;
          bool near = false;
          for (size_t r = 0; r < rx.size() && !near; r++) {
            const double gx = axis_gap(rx[r], ci * s, (ci + 1) * s, Lx), gy = axis_gap(ry[r], cj * s, (cj + 1) * s, Ly);
            near = std::sqrt(gx * gx + gy * gy) <= s;
          }
          if (near) T.refined[l][T.idx(l, ci, cj, ck)] = 1;
        }
    }
  }
  // the level of the leaf covering the region of cube (ci, cj, ck) of level l,
  // and that leaf's index
  auto leaf_of = [&](int l, int ci, int cj, int ck, int &m, int &mi, int &mj, int &mk) {
    const long long f = 1LL << (L - l);
    const long long px = (2LL * ci + 1) * f, py = (2LL * cj + 1) * f, pz = (2LL * ck + 1) * f;
    for (m = 0; m < nlev; m++) {
      const long long g = 1LL << (L - m + 1);
      mi = (int)(px / g);
      mj = (int)(py / g);
      mk = (int)(pz / g);
      if (!T.is_ref(m, mi, mj, mk)) return;
    }
  };
  // 2:1 balance across faces, edges and corners (periodic in x and y)
  bool changed = true;
  while (changed) {
    changed = false;
    for (int l = L; l >= 2; l--)
      for (int pk = 0; pk < T.ncz[l - 1]; pk++)
        for (int pj = 0; pj < T.ncy[l - 1]; pj++)
          for (int pi = 0; pi < T.ncx[l - 1]; pi++) {
            if (!T.is_ref(l - 1, pi, pj, pk)) continue;
            for (int e = 0; e < 8; e++) {
              const int ci = 2 * pi + (e & 1), cj = 2 * pj + ((e >> 1) & 1), ck = 2 * pk + (e >> 2);
              if (T.is_ref(l, ci, cj, ck)) continue;
              for (int dk = -1; dk <= 1; dk++)
                for (int dj = -1; dj <= 1; dj++)
                  for (int di = -1; di <= 1; di++) {
                    if (!di && !dj && !dk) continue;
                    const int nk = ck + dk;
                    if (nk < 0 || nk >= T.ncz[l]) continue;
                    const int ni = (ci + di + T.ncx[l]) % T.ncx[l], nj = (cj + dj + T.ncy[l]) % T.ncy[l];
                    int m, mi, mj, mk;
                    leaf_of(l, ni, nj, nk, m, mi, mj, mk);
                    if (m < l - 1) {
                      T.refined[m][T.idx(m, mi, mj, mk)] = 1;
                      changed = true;
                    }
                  }
            }
          }
  }
  // leaves, minus the cubes completely inside the terrain, by (level, ck, cj, ci)
  int n = 0;
  for (int l = 0; l < nlev; l++) {
    const double s = size(l);
    const long long f = (long long)cube << (L - l);
    for (int ck = 0; ck < T.ncz[l]; ck++)
      for (int cj = 0; cj < T.ncy[l]; cj++)
        for (int ci = 0; ci < T.ncx[l]; ci++) {
          if (!T.exists(l, ci, cj, ck) || T.is_ref(l, ci, cj, ck)) continue;
          double lo = 1e300;
          for (long long J = cj * f; J <= (cj + 1) * f; J++)
            for (long long I = ci * f; I <= (ci + 1) * f; I++) lo = std::min(lo, h_finest[(J % fny) * fnx + (I % fnx)]);
          if (lo >= (ck + 1) * s) continue;
          if (out && n < capacity) out[n] = cc_cube{l, ci, cj, ck};
          n++;
        }
  }
  *count = n;
  return (out && n > capacity) ? CC_EINVAL : CC_OK;
}
