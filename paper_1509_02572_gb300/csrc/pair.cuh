// The full-cell stencil in FP32 with two x-adjacent cells per thread
// (included by step.cu, after k_full, whose helpers it uses).
//
// The same step as k_full (Sec 2.4: aperture-weighted face fluxes and their
// divergence, the p' and rho' tendencies, the momentum equations
// momentum_u_d .. momentum_w_d, the artificial diffusion of Sec 2.1 with the
// wall-aware form of Sec 2.4, sponge, leapfrog and Robert-Asselin filter),
// each thread taking the cells (i, j, k) and (i + 1, j, k), i even, and their
// corners.  Two adjacent cells are two adjacent values of a shared-memory row,
// so one 8-byte load feeds both and the arithmetic runs on float2 pairs
// (packed FP32: every lane is rounded as the scalar operation would be).  The
// face fluxes, corner densities, corner velocities and equation of state are
// the scalar kernels' operations in their order, so a face this kernel shares
// with a cut cell or a refined box has the same bits on both sides.  The
// x-face between this thread's pair and the next thread's is computed once,
// by the next thread, and passed with a warp shuffle.
//
// Staging, by domain: two instantiations, each launched over its part of the
// work list.  k_pair<TY, true> takes the tiles of refined boxes, whose haloed
// planes lie inside the padded arrays: one thread moves each plane with TMA
// box copies (cp.async.bulk.tensor; one tensor map per domain over its twenty
// padded field arrays, which lie back to back), completing on an mbarrier per
// plane in flight, on whose phase the other threads wait.  The box starts two
// columns left of the tile, on a 16-byte boundary (tiles start at multiples
// of 4 and the padding is 6 columns); points past the padding arrive as
// zeros, which no computed point reads.  k_pair<TY, false> takes the tiles of
// periodic domains, whose halos wrap at the lateral edges (a box cannot), and
// gathers each plane with per-thread 16-byte cp.async copies from the cyclic
// indices.  Measured alternatives for the periodic tiles, all slower than the
// gather: a ghost frame kept current by the writers or by a copy kernel, the
// two paths mixed in one launch, and the seam tiles in a launch of their own.

__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
// the one arrival of a plane's barrier, with the bytes its copies will bring
__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;\n" : "=l"(t));
  return t;
}
// waits for the phase of the given parity to complete; false after limit_ns
// without completion (the caller reports it and stops)
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned parity, unsigned long long limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  while (!mbar_try_wait(bar, parity))
    if (global_ns() - t0 > limit_ns) return false;
  return true;
}
constexpr unsigned long long PAIR_WAIT_NS = 1000000000ull;  // a plane's copies: one second
constexpr unsigned long long PAIR_DRAIN_NS = 250000000ull;  // after an abort, per plane in flight
// box copy of the tensor map's box at (x, y, z) into dst, completing on bar
__device__ __forceinline__ void tma_load3(void *dst, const void *tmap, unsigned long long *bar, int x, int y, int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];\n" ::"r"(smem_u32(dst)),
      "l"(tmap), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ float2 bc2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
// a - b as fma(b, -1, a): one rounding, the same value as the rounded difference
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 ld2(const float *p) { return *reinterpret_cast<const float2 *>(p); }
__device__ __forceinline__ void st2(float *p, float2 v) { *reinterpret_cast<float2 *>(p) = v; }
// the pair (p[-1], p[0]) from the aligned pairs at p - 2 and p
__device__ __forceinline__ float2 odd2(float2 lo, float2 hi) { return make_float2(lo.y, hi.x); }

__device__ __forceinline__ float2 face_flux2(float2 pa, float2 pb, float2 un, float2 S) {
  return mul2(mul2(mul2(add2(pa, pb), bc2(0.5f)), un), S);
}
__device__ __forceinline__ float2 mean4(float2 u1, float2 u2, float2 u3, float2 u4) {
  return mul2(add2(add2(u1, u2), add2(u3, u4)), bc2(0.25f));
}
__device__ __forceinline__ float2 rho8_2(float2 a, float2 b, float2 c, float2 d, float2 e, float2 f, float2 g,
                                         float2 h) {
  return mul2(add2(add2(add2(a, b), add2(c, d)), add2(add2(e, f), add2(g, h))), bc2(0.125f));
}
__device__ __forceinline__ float2 rinv2(float2 r) { return make_float2(rinv(r.x), rinv(r.y)); }

// (1 + x)^a - 1 for a pair: the binomial series of pow1pm1_e on both lanes
// when both are small, else lane by lane
__device__ __forceinline__ float2 pow1pm1_2(float2 x, const float (&c)[8]) {
  if (fabsf(x.x) < 0.0625f && fabsf(x.y) < 0.0625f) {
    float2 s = bc2(c[6]);
    s = fma2(s, x, bc2(c[5]));
    s = fma2(s, x, bc2(c[4]));
    s = fma2(s, x, bc2(c[3]));
    s = fma2(s, x, bc2(c[2]));
    s = fma2(s, x, bc2(c[1]));
    s = fma2(s, x, bc2(c[0]));
    return mul2(s, x);
  }
  return make_float2(pow1pm1_e(x.x, c), pow1pm1_e(x.y, c));
}
struct EosK2 {
  float thb, ipb, pik;
  __device__ __forceinline__ void load(const float *thb_, const float *ipb_, const float *pik_, int kp) {
    thb = thb_[kp];
    ipb = ipb_[kp];
    pik = pik_[kp];
  }
  __device__ __forceinline__ float2 pert(const Eos &E, float2 pp) const {
    return mul2(bc2(thb), pow1pm1_2(mul2(pp, bc2(ipb)), E.sth));
  }
  __device__ __forceinline__ float2 tot(const Eos &E, float2 pp) const { return add2(bc2(thb), pert(E, pp)); }
  __device__ __forceinline__ float2 exner(const Eos &E, float2 pp) const {
    return fma2(bc2(pik), pow1pm1_2(mul2(pp, bc2(ipb)), E.sex), bc2(pik));
  }
};

// the diffusion sum of one axis for a pair, lane by lane (diff_axis)
__device__ __forceinline__ float2 dax2(float2 a, float2 b, float2 c, float2 d, float2 e, bool scalar, const bool (&f0)[4],
                                       const bool (&f1)[4]) {
  return make_float2(diff_axis(a.x, b.x, c.x, d.x, e.x, f0[0], f0[1], f0[2], f0[3], scalar),
                     diff_axis(a.y, b.y, c.y, d.y, e.y, f1[0], f1[1], f1[2], f1[3], scalar));
}
__device__ __forceinline__ float2 d4_2(float2 a, float2 b, float2 c, float2 d, float2 e) {
  return make_float2(d4(a.x, b.x, c.x, d.x, e.x), d4(a.y, b.y, c.y, d.y, e.y));
}

// NR warp roles: 1, every thread updates the scalars and the momenta of its
// pair; 2, the block holds two warpgroups of NT threads over the same tile,
// the first updating rho' and p', the second the three momenta (the two
// updates read the same staged planes and nothing of each other), so that
// each thread holds the live values of one update only and twice as many
// warps fit per SM.  The staging and the derived planes are shared out over
// all NR NT threads.
template <bool B>
struct RoleTag {
  static constexpr bool value = B;
};

template <int TYv, int NR = 1>
struct PairCfg {
  static constexpr int TX = TILE_X, TY = TYv, NT = (TILE_X / 2) * TYv, NTH = NR * NT, HX = TX + 4, HY = TYv + 4,
                       PL = HX * HY, NPP = PL / 2, NLPP = (NPP + NTH - 1) / NTH;
  // pitch of a raw plane slot: whole 128-byte lines, so that every TMA
  // destination is 128-byte aligned
  static constexpr int PLP = (PL + 31) / 32 * 32;
};

// planes in flight at most: five at the start of a column, one per plane after
constexpr int PAIR_NBAR = 8;

// shared memory of k_pair: the rings of FullSmem, raw slots padded to whole
// 128-byte lines, and the plane barriers
template <int PL, int PLP>
struct PairSmem {
  float cr[5][PLP], cp[5][PLP];  // raw rho', p' (current level), planes k-1 .. k+3
  float cm[4][3][PLP];           // raw momentum (current level), planes k-1 .. k+2 (+ in flight)
  float op[4][PLP];              // raw p' at n-1, planes k .. k+3
  float om[4][3][PLP];           // raw momentum at n-1, planes k .. k+3
  float rh[4][PL], th[4][PL];    // total density and total rho theta, planes k-1 .. k+2
  float uu[3][3][PL];            // corner velocity, planes k-1 .. k+1
  float to[PL];                  // (rho theta)' at n-1, plane k
  unsigned long long bar[PAIR_NBAR];
  int abort;
};

// TMA: the tiles of the work list are staged with TMA box copies; otherwise
// (periodic tiles whose halo crosses a lateral edge) by the cyclic gather
// NR = 2 takes 128 registers per thread at most: two blocks of 8 warps per SM
// for 32x8 tiles, one of 16 warps for 32x16 tiles
template <int TYv, bool TMA, int NR>
__global__ void __launch_bounds__(NR *(TILE_X / 2) * TYv, NR == 2 && TYv == 8 ? 2 : 1)
    k_pair(const DomDev *__restrict__ doms, const WorkItem *__restrict__ items, const unsigned char *__restrict__ tmaps,
           int rO, int rC, int rN, int rF, int first, const Eos E, unsigned *__restrict__ watch,
           unsigned stall_tx) {
  using C = PairCfg<TYv, NR>;
  constexpr int NT = C::NT, NTH = C::NTH, HX = C::HX, PL = C::PL, PLP = C::PLP, NPP = C::NPP, NLPP = C::NLPP;
  static_assert(HX % 4 == 0, "halo rows of whole 16-byte chunks");
  extern __shared__ __align__(128) unsigned char smraw[];
  // TMA: the rings start on a 128-byte line (the launch adds 128 bytes for
  // this) and their raw slots are whole lines
  using Smem = PairSmem<PL, TMA ? PLP : PL>;
  Smem &S = *reinterpret_cast<Smem *>(smraw + (TMA ? ((128u - (smem_u32(smraw) & 127u)) & 127u) : 0u));
  const WorkItem W = items[blockIdx.x];
  const DomDev &D = doms[W.dom];
  // this domain's tensor map for this tile height (two 128-byte maps per domain)
  const void *tmap = tmaps + (2 * W.dom + (TYv == 16 ? 1 : 0)) * 128;
  const float dt2 = (float)(first ? D.dt : 2.0 * D.dt);
  const float nu = (float)(first ? 0.0 : D.ra_nu);
  const int tid = threadIdx.x;
  const int nx = D.nx, ny = D.ny, nz = D.nz, px = D.px;
  const long long plane = D.plane;
  const float *__restrict__ rpC = (const float *)D.f[rC][0];
  const float *__restrict__ ppC = (const float *)D.f[rC][1];
  const float *__restrict__ mC0 = (const float *)D.f[rC][2];
  const float *__restrict__ mC1 = (const float *)D.f[rC][3];
  const float *__restrict__ mC2 = (const float *)D.f[rC][4];
  const float *__restrict__ rpO = (const float *)D.f[rO][0];
  const float *__restrict__ ppO = (const float *)D.f[rO][1];
  const float *__restrict__ mO0 = (const float *)D.f[rO][2];
  const float *__restrict__ mO1 = (const float *)D.f[rO][3];
  const float *__restrict__ mO2 = (const float *)D.f[rO][4];
  float *__restrict__ rpN = (float *)D.f[rN][0];
  float *__restrict__ ppN = (float *)D.f[rN][1];
  float *__restrict__ rpF = (float *)D.f[rF][0];
  float *__restrict__ ppF = (float *)D.f[rF][1];
  float *__restrict__ mN[3] = {(float *)D.f[rN][2], (float *)D.f[rN][3], (float *)D.f[rN][4]};
  float *__restrict__ mF[3] = {(float *)D.f[rF][2], (float *)D.f[rF][3], (float *)D.f[rF][4]};
  const float *__restrict__ rhob = (const float *)D.rhob;
  const float *__restrict__ ipb = (const float *)D.ipb;
  const float *__restrict__ thb = (const float *)D.thb;
  const float *__restrict__ pik = (const float *)D.pik;
  const float *__restrict__ rhobc = (const float *)D.rhobc;
  const float *__restrict__ tau = (const float *)D.tau;
  const int i0 = W.i0, j0 = W.j0, k0 = W.k0, k1 = W.k1;

  auto col_x = [&](int gi) { return D.periodic ? wrapi(gi, nx) : min(max(gi, -GX), px - GX - 1); };
  auto row_y = [&](int gj) { return D.periodic ? wrapi(gj, ny) : min(max(gj, -GH), D.py - GH - 1); };
  // pairs of halo points this thread derives: points 2 pp and 2 pp + 1, pp =
  // s NTH + hpair; with two roles the warps of the two warpgroups take runs of
  // 32 pairs in turn, so that both share the derived planes about evenly
  const int hpair = NR == 1 ? tid : (2 * ((tid % NT) >> 5) + tid / NT) * 32 + (tid & 31);
  int loff[NLPP][2], kbv[NLPP][2];
#pragma unroll
  for (int s = 0; s < NLPP; s++) {
    const int pp = s * NTH + hpair;
#pragma unroll
    for (int h = 0; h < 2; h++) {
      const int p = 2 * pp + h;
      const int hx = p % HX, hy = p / HX;
      loff[s][h] = (row_y(j0 - 2 + hy) + GH) * px + (col_x(i0 - 2 + hx) + GX);
      kbv[s][h] = pp < NPP ? D.kb[loff[s][h]] : KB_NONE;
    }
  }
  const float *__restrict__ ubC = (const float *)D.ub[rC];
  const int kmaxp = D.pz - GH - 1;  // highest plane inside the padding
  // TMA coordinates: box origin (padded x and y of the halo's first point);
  // z runs over the twenty arrays, level b field f at (b NFIELD + f) pz
  const int bx = i0 - 2 + GX, by = j0 - 2 + GH, pz = D.pz;
  const int zC = rC * NFIELD * pz, zO = rO * NFIELD * pz;
  // the copies of plane kk (thread 0): the current-level momentum when with_m,
  // the n-1 fields when with_o; planes past the top are never used
  auto issue = [&](int kk, bool with_m, bool with_o) {
    const int zc = min(kk, kmaxp) + GH;
    unsigned long long *bar = &S.bar[(kk - (k0 - 2)) & (PAIR_NBAR - 1)];
    // (stall_tx, zero but in the watchdog's test, makes the phase wait for
    // bytes that never come)
    mbar_expect_tx(bar, (unsigned)((2 + (with_m ? 3 : 0) + (with_o ? 4 : 0)) * PL * sizeof(float)) + stall_tx);
    const int a5 = s5(kk), a4 = s4(kk);
    tma_load3(S.cr[a5], tmap, bar, bx, by, zC + zc);
    tma_load3(S.cp[a5], tmap, bar, bx, by, zC + pz + zc);
    if (with_m) {
#pragma unroll
      for (int d = 0; d < 3; d++) tma_load3(S.cm[a4][d], tmap, bar, bx, by, zC + (2 + d) * pz + zc);
    }
    if (with_o) {
      tma_load3(S.op[a4], tmap, bar, bx, by, zO + pz + zc);
#pragma unroll
      for (int d = 0; d < 3; d++) tma_load3(S.om[a4][d], tmap, bar, bx, by, zO + (2 + d) * pz + zc);
    }
  };
  // every thread waits for the copies of plane kk; a wait that runs out
  // marks the block for abort, and the thread waits no more
  bool late = false;
  auto wait_plane = [&](int kk) {
    const int u = kk - (k0 - 2);
    if (late) return;
    if (!mbar_wait(&S.bar[u & (PAIR_NBAR - 1)], (unsigned)(u / PAIR_NBAR) & 1u, PAIR_WAIT_NS)) {
      late = true;
      S.abort = 1;
    }
  };
  // a periodic tile whose halo crosses a lateral edge: 16-byte chunks of the
  // haloed rows from the cyclic indices, element by element where a chunk
  // crosses the edge
  // (NT threads: with two roles those of the momentum warpgroup, and the
  // scalar warpgroup holds no copy state; measured 3 % faster on the
  // 64-instance ensemble than the copies on the scalar side)
  constexpr int VEC = 4, CPR = HX / VEC, NCH = CPR * C::HY, NCQ = (NCH + NT - 1) / NT;
  int ch_dst[NCQ], ch_e[NCQ][VEC];
  bool ch_whole[NCQ];
#pragma unroll
  for (int q = 0; q < NCQ; q++) {
    const int t = tid % NT + q * NT;
    const int row = t / CPR, col = t % CPR;
    const int x = i0 - 2 + VEC * col;
    const int rowoff = (row_y(j0 - 2 + row) + GH) * px;
    ch_dst[q] = !TMA && (NR == 1 || tid >= NT) && t < NCH ? row * HX + VEC * col : -1;
    ch_whole[q] = x >= 0 && x + VEC <= nx;
#pragma unroll
    for (int e = 0; e < VEC; e++) ch_e[q][e] = rowoff + col_x(x + e) + GX;
  }
  auto chunk = [&](float *dst, const float *src) {
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
  auto gather = [&](int kk, bool with_m, bool with_o) {
    const long long zo = (long long)(min(kk, kmaxp) + GH) * plane;
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
    acommit();
  };
  // the copies of plane kk by the path of this kernel, and the wait for them
  auto stage = [&](int kk, bool with_m, bool with_o) {
    if constexpr (TMA) {
      if (tid == 0) issue(kk, with_m, with_o);
    } else {
      gather(kk, with_m, with_o);
    }
  };
  auto arrive = [&](int kk) {
    if constexpr (TMA)
      wait_plane(kk);
    else
      await_groups<0>();
  };
  // totals of plane kk (pairs of halo points)
  auto derive_e = [&](int kk, const float rb, const EosK2 ek) {
    const float *cr = S.cr[s5(kk)], *cp = S.cp[s5(kk)];
    float *rh = S.rh[s4(kk)], *th = S.th[s4(kk)];
#pragma unroll
    for (int s = 0; s < NLPP; s++) {
      const int pp = s * NTH + hpair;
      if (pp < NPP) {
        const int p = 2 * pp;
        st2(rh + p, add2(bc2(rb), ld2(cr + p)));
        st2(th + p, ek.tot(E, ld2(cp + p)));
      }
    }
  };
  auto derive = [&](int kk) {
    EosK2 ek;
    ek.load(thb, ipb, pik, kk + GH);
    derive_e(kk, rhob[kk + GH], ek);
  };
  // corner velocities of plane K, two corners at a time; a corner at or below
  // the terrain takes the boundary-point velocity of its column
  auto velocity = [&](int K) {
    const float *lo = S.rh[s4(K - 1)], *hi = S.rh[s4(K)];
    const int su = s3(K), sm = s4(K);
#pragma unroll
    for (int s = 0; s < NLPP; s++) {
      const int pp = s * NTH + hpair;
      const int p = 2 * pp;
      const int hx = p % HX, hy = p / HX;
      if (pp < NPP && hy != 0) {
        // corner p needs cells p-HX-1, p-HX, p-1, p; corner p+1 cells p-HX .. p+1.  On the
        // halo's first column (hx = 0) the corner p is never used: read the pair at p instead
        const int am = hx == 0 ? 0 : 2;
        const float2 A0 = ld2(lo + p - HX - am), B0 = ld2(lo + p - HX), C0 = ld2(lo + p - am), D0 = ld2(lo + p);
        const float2 A1 = ld2(hi + p - HX - am), B1 = ld2(hi + p - HX), C1 = ld2(hi + p - am), D1 = ld2(hi + p);
        const float2 iv = rinv2(rho8_2(odd2(A0, B0), B0, odd2(C0, D0), D0, odd2(A1, B1), B1, odd2(C1, D1), D1));
        float2 u0 = mul2(ld2(S.cm[sm][0] + p), iv), u1 = mul2(ld2(S.cm[sm][1] + p), iv),
               u2 = mul2(ld2(S.cm[sm][2] + p), iv);
        if (K <= kbv[s][0] || K <= kbv[s][1]) {
          if (K <= kbv[s][0]) {
            const float *u = ubC + 3 * loff[s][0];
            u0.x = u[0];
            u1.x = u[1];
            u2.x = u[2];
          }
          if (K <= kbv[s][1]) {
            const float *u = ubC + 3 * loff[s][1];
            u0.y = u[0];
            u1.y = u[1];
            u2.y = u[2];
          }
        }
        st2(S.uu[su][0] + p, u0);
        st2(S.uu[su][1] + p, u1);
        st2(S.uu[su][2] + p, u2);
      }
    }
  };
  auto derive_old_e = [&](int kk, const EosK2 ek) {
    const float *op = S.op[s4(kk)];
#pragma unroll
    for (int s = 0; s < NLPP; s++) {
      const int pp = s * NTH + hpair;
      if (pp < NPP) st2(S.to + 2 * pp, ek.pert(E, ld2(op + 2 * pp)));
    }
  };

  // the pair of this thread (both warpgroups of NR = 2 map onto the tile's NT
  // pairs alike) and its role
  const int lt = NR == 1 ? tid : tid % NT;
  const int role = NR == 1 ? 0 : tid / NT;  // NR = 2: 0 the scalars, 1 the momenta
  const int tx = lt & 15, ty = lt >> 4;
  const int i = i0 + 2 * tx, j = j0 + ty;
  const bool rowok = j < D.cj1;
  const bool a0 = rowok && i >= D.ci0 && i < D.ci1, a1 = rowok && i + 1 >= D.ci0 && i + 1 < D.ci1;
  const bool active = a0 || a1;
  // corners of a refined box outside -1 .. n+1 are ghost values from the coarser level
  const bool q0 = a0 && i >= D.qi0 && j >= D.qj0, q1 = a1 && i + 1 >= D.qi0 && j >= D.qj0;
  const int c = (ty + 2) * HX + (2 * tx + 2);
  const long long own = active ? (long long)(j + GH) * px + (i + GX) : 0;
  const float qdx = (float)(0.25 / D.dx), qdy = (float)(0.25 / D.dy), qdz = (float)(0.25 / D.dz);
  const float2 Sx = bc2((float)(D.dy * D.dz)), Sy = bc2((float)(D.dx * D.dz)), Sz = bc2((float)(D.dx * D.dy));
  const float hSx = (float)(0.25 * D.dy * D.dz), hSy = (float)(0.25 * D.dx * D.dz), hSz = (float)(0.25 * D.dx * D.dy);
  const float v0inv = (float)(1.0 / (D.dx * D.dy * D.dz));
  const float kdif = (float)D.kdif, Cp = (float)D.Cp, g = (float)D.g, U = (float)D.U;
  const int kug0 = a0 ? D.kug[own] : 0, kug1 = a1 ? D.kug[own + 1] : 0;
  const int dlo = active ? max(a0 ? (int)D.dcol[own].lo : -1000, a1 ? (int)D.dcol[own + 1].lo : -1000) : 0;
  const int dhi = active ? min(a0 ? (int)D.dcol[own].hi : 1000000, a1 ? (int)D.dcol[own + 1].hi : 1000000) : 0;
  const bool last_tx = tx == 15;

  // own columns at n-1 for the vertical diffusion stencils, levels k-2 .. k+2
  float2 treg[5], mreg[5][3];
  auto own_old_e = [&](int a, int kk, const EosK2 ek) {
    const int a4 = s4(kk);
    treg[a] = ek.pert(E, ld2(S.op[a4] + c));
    mreg[a][0] = ld2(S.om[a4][0] + c);
    mreg[a][1] = ld2(S.om[a4][1] + c);
    mreg[a][2] = ld2(S.om[a4][2] + c);
  };

  // the barrier of the z-march: with two roles the warpgroups run separate
  // code, so a named barrier over all NTH threads (warps may reach it from
  // different places)
  auto sync_all = [] {
    if constexpr (NR == 1)
      __syncthreads();
    else
      asm volatile("bar.sync 1, %0;\n" ::"r"(NTH) : "memory");
  };
  // a TMA wait that ran out (the same answer in every thread after a barrier)
  auto aborted = [&] {
    if constexpr (TMA)
      return S.abort != 0;
    else
      return false;
  };
  if constexpr (TMA) {
    if (tid == 0) {
      for (int b = 0; b < PAIR_NBAR; b++) mbar_init(&S.bar[b], 1);
      S.abort = 0;
      asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
      asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    }
    __syncthreads();
  }
  for (int kk = k0 - 2; kk <= k0 + 2; kk++) stage(kk, kk != k0 - 2, kk != k0 - 2);
  int issued = k0 + 2;  // last plane whose copies were issued
  {
    const long long o2 = (long long)(k0 - 2 + GH) * plane + own;
    EosK2 ek;
    ek.load(thb, ipb, pik, k0 - 2 + GH);
    treg[0] = ek.pert(E, ld2(ppO + o2));
    mreg[0][0] = ld2(mO0 + o2);
    mreg[0][1] = ld2(mO1 + o2);
    mreg[0][2] = ld2(mO2 + o2);
  }
  for (int kk = k0 - 2; kk <= k0 + 2; kk++) arrive(kk);
  __syncthreads();
  // after an abort the set-up below runs on whatever the rings hold (shared
  // memory only) and the z-march, the one writer of global memory, is skipped
  const bool started = !aborted();
  for (int kk = k0 - 2; kk <= k0 + 1; kk++) derive(kk);
#pragma unroll
  for (int a = 1; a < 4; a++) {
    EosK2 ek;
    ek.load(thb, ipb, pik, k0 - 2 + a + GH);
    own_old_e(a, k0 - 2 + a, ek);
  }
  __syncthreads();
  velocity(k0 - 1);
  velocity(k0);

  const float cfx = (float)(D.dt / D.dx), cfy = (float)(D.dt / D.dy), cfz = (float)(D.dt / D.dz);
  // the z-march of this thread's role: DS the scalar update, DM the momentum
  // update (both when NR = 1); returns the watchdog flags
  auto march = [&](auto ds_, auto dm_) -> unsigned {
    constexpr bool DS = decltype(ds_)::value, DM = decltype(dm_)::value;
    float2 fz_carry = bc2(0.0f), hz_carry = bc2(0.0f);
    unsigned wflag = 0;
    for (int k = k0; started && k < k1; k++) {
      const long long o = (long long)(k + GH) * plane + own;
      float2 rO_ = bc2(0.0f);
      if (DS && active) rO_ = ld2(rpO + o);
      EosK2 ek0, ek2;
      ek0.load(thb, ipb, pik, k + GH);
      ek2.load(thb, ipb, pik, k + 2 + GH);
      const float rb2 = rhob[k + 2 + GH];
      float tk = 0.0f, rbc[5] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
      if constexpr (DM) {
        tk = tau[k + GH];
#pragma unroll
        for (int a = 0; a < 5; a++) rbc[a] = rhobc[k + GH - 2 + a] * U;
      }
      arrive(k + 2);
      sync_all();
      if (aborted()) break;
      // plane k + 3 is read from the next plane on; the last plane needs k1 + 1
      // (TMA: thread 0, in the scalar role; gather: the momentum role's threads)
      if ((TMA ? DS : DM) && k + 3 <= k1 + 1) {
        stage(k + 3, true, true);
        issued = k + 3;
      }
      derive_e(k + 2, rb2, ek2);
      velocity(k + 1);
      derive_old_e(k, ek0);
      if constexpr (DS) treg[4] = ek2.pert(E, ld2(S.op[s4(k + 2)] + c));
      if constexpr (DM && NR == 1) {
        const int a4 = s4(k + 2);
        mreg[4][0] = ld2(S.om[a4][0] + c);
        mreg[4][1] = ld2(S.om[a4][1] + c);
        mreg[4][2] = ld2(S.om[a4][2] + c);
      }
      // the own column's momentum at n-1, level k - 2 + a: one role keeps all
      // five levels in registers; the momentum role of two keeps levels k-2
      // and k-1 and reads k .. k+2 from the ring, which still holds them
      auto mo = [&](int a, int d) -> float2 {
        if constexpr (NR == 2)
          if (a >= 2) return ld2(S.om[s4(k - 2 + a)][d] + c);
        return mreg[a][d];
      };
      sync_all();
      // the x-faces: this thread's low faces (i - 1/2, i + 1/2) as a pair; its
      // highest face (i + 3/2) is the next thread's lowest, taken by shuffle
      const int sk = s4(k), skm = s4(k - 1), skp = s4(k + 1);
      const int ck = s5(k), ckm = s5(k - 1);
      const float *R0 = S.rh[sk], *Rm = S.rh[skm], *Rp = S.rh[skp];
      const float *H0 = S.th[sk], *Hm = S.th[skm], *Hp = S.th[skp];
      const int uk = s3(k), ukp = s3(k + 1), ukm = s3(k - 1);
      const float *ux0 = S.uu[uk][0], *uy0 = S.uu[uk][1], *uz0 = S.uu[uk][2];
      const float *uxp = S.uu[ukp][0], *uyp = S.uu[ukp][1], *uzp = S.uu[ukp][2];
      const float2 Rc = ld2(R0 + c), Rl = ld2(R0 + c - 2);
      float2 Hc = bc2(0.0f), fxl = bc2(0.0f), hxl = bc2(0.0f);
      float fxh = 0.0f, hxh = 0.0f;
      if constexpr (DS) {
        Hc = ld2(H0 + c);
        const float2 Hl = ld2(H0 + c - 2);
        const float2 unx = mean4(ld2(ux0 + c), ld2(ux0 + c + HX), ld2(uxp + c), ld2(uxp + c + HX));
        fxl = face_flux2(odd2(Rl, Rc), Rc, unx, Sx);
        hxl = face_flux2(odd2(Hl, Hc), Hc, unx, Sx);
        fxh = __shfl_down_sync(0xffffffffu, fxl.x, 1);
        hxh = __shfl_down_sync(0xffffffffu, hxl.x, 1);
        if (last_tx) {
          // the tile's last face, from the halo
          const float r2 = R0[c + 2], h2 = H0[c + 2];
          const float un = Ar<float>::mul(Ar<float>::add(Ar<float>::add(ux0[c + 2], ux0[c + 2 + HX]),
                                                         Ar<float>::add(uxp[c + 2], uxp[c + 2 + HX])),
                                          0.25f);
          fxh = Ar<float>::mul(Ar<float>::mul(Ar<float>::mul(Ar<float>::add(Rc.y, r2), 0.5f), un), Sx.x);
          hxh = Ar<float>::mul(Ar<float>::mul(Ar<float>::mul(Ar<float>::add(Hc.y, h2), 0.5f), un), Sx.x);
        }
      }
      if (active) {
        const float2 RS = ld2(R0 + c - HX);
        float2 RM = bc2(0.0f), RH = bc2(0.0f);
        if constexpr (DS) {
        const float2 fxm = fxl, fxp = make_float2(fxl.y, fxh);
        const float2 hxm = hxl, hxp = make_float2(hxl.y, hxh);
        // y-faces: the corners (c, c+1) of cell c and (c+1, c+2) of cell c+1
        const float2 uy00 = ld2(uy0 + c), uy02 = ld2(uy0 + c + 2), uyp0 = ld2(uyp + c), uyp2 = ld2(uyp + c + 2);
        const float2 uy0H = ld2(uy0 + c + HX), uy0H2 = ld2(uy0 + c + HX + 2), uypH = ld2(uyp + c + HX),
                     uypH2 = ld2(uyp + c + HX + 2);
        const float2 unym = mean4(uy00, odd2(uy00, uy02), uyp0, odd2(uyp0, uyp2));
        const float2 unyp = mean4(uy0H, odd2(uy0H, uy0H2), uypH, odd2(uypH, uypH2));
        const float2 RN = ld2(R0 + c + HX), HS = ld2(H0 + c - HX), HN = ld2(H0 + c + HX);
        const float2 fym = face_flux2(RS, Rc, unym, Sy), fyp = face_flux2(Rc, RN, unyp, Sy);
        const float2 hym = face_flux2(HS, Hc, unym, Sy), hyp = face_flux2(Hc, HN, unyp, Sy);
        // z-faces: corners (c, c+1, c+HX, c+HX+1) of the upper face; the lower
        // face is the one of the plane below
        const float2 uzp0 = ld2(uzp + c), uzp2 = ld2(uzp + c + 2), uzpH = ld2(uzp + c + HX),
                     uzpH2 = ld2(uzp + c + HX + 2);
        const float2 unzp = mean4(uzp0, odd2(uzp0, uzp2), uzpH, odd2(uzpH, uzpH2));
        float2 fzp = face_flux2(Rc, ld2(Rp + c), unzp, Sz), hzp = face_flux2(Hc, ld2(Hp + c), unzp, Sz);
        float2 fzm = fz_carry, hzm = hz_carry;
        if (k == k0) {
          const float2 uz00 = ld2(uz0 + c), uz02 = ld2(uz0 + c + 2), uz0H = ld2(uz0 + c + HX),
                       uz0H2 = ld2(uz0 + c + HX + 2);
          const float2 unzm = mean4(uz00, odd2(uz00, uz02), uz0H, odd2(uz0H, uz0H2));
          fzm = face_flux2(ld2(Rm + c), Rc, unzm, Sz);
          hzm = face_flux2(ld2(Hm + c), Hc, unzm, Sz);
        }
        fz_carry = fzp;
        hz_carry = hzp;
        if (k == 0) {
          fzm = bc2(0.0f);
          hzm = bc2(0.0f);
        }
        if (D.lid && k == nz - 1) {
          fzp = bc2(0.0f);
          hzp = bc2(0.0f);
        }
        RM = add2(add2(sub2(fxp, fxm), sub2(fyp, fym)), sub2(fzp, fzm));
        RH = add2(add2(sub2(hxp, hxm), sub2(hyp, hym)), sub2(hzp, hzm));
        }

        // ---- artificial diffusion at n-1
        const int ok4 = s4(k);
        const bool wall = k < dlo || k >= dhi;
        float2 dd = bc2(0.0f), dmv[3] = {bc2(0.0f), bc2(0.0f), bc2(0.0f)};
        // the momentum sums of one component d, with the axis sum f (fourth
        // difference or wall-aware form) and the vertical flags gz
        auto dmom = [&](int d, auto f) {
          const float *Mk = S.om[ok4][d];
          const float2 ref0 = bc2(d == 0 ? rbc[2] : 0.0f);
          const float2 m2 = sub2(ld2(Mk + c - 2), ref0), m0 = sub2(ld2(Mk + c), ref0), p2 = sub2(ld2(Mk + c + 2), ref0);
          const float2 l1 = odd2(m2, m0), r1 = odd2(m0, p2);
          float2 dm = add2(f(0, m2, l1, m0, r1, p2),
                           f(1, sub2(ld2(Mk + c - 2 * HX), ref0), sub2(ld2(Mk + c - HX), ref0), m0,
                             sub2(ld2(Mk + c + HX), ref0), sub2(ld2(Mk + c + 2 * HX), ref0)));
          if (d == 0)
            dm = add2(dm, f(2, sub2(mo(0, 0), bc2(rbc[0])), sub2(mo(1, 0), bc2(rbc[1])), sub2(mo(2, 0), ref0),
                            sub2(mo(3, 0), bc2(rbc[3])), sub2(mo(4, 0), bc2(rbc[4]))));
          else
            dm = add2(dm, f(2, mo(0, d), mo(1, d), mo(2, d), mo(3, d), mo(4, d)));
          return dm;
        };
        if (!wall) {
          auto f4 = [](int, float2 a, float2 b, float2 c_, float2 d, float2 e) { return d4_2(a, b, c_, d, e); };
          if constexpr (DS) {
            const float *Tk = S.to;
            const float2 Tm2 = ld2(Tk + c - 2), Tc = ld2(Tk + c), Tp2 = ld2(Tk + c + 2);
            const float2 Tl = odd2(Tm2, Tc), Tr = odd2(Tc, Tp2);
            const float2 TS2 = ld2(Tk + c - 2 * HX), TS = ld2(Tk + c - HX), TN = ld2(Tk + c + HX),
                         TN2 = ld2(Tk + c + 2 * HX);
            // x stencil of the pair: (c-2, c-1, c, c+1, c+2) and (c-1, c, c+1, c+2, c+3)
            dd = add2(add2(d4_2(Tm2, Tl, Tc, Tr, Tp2), d4_2(TS2, TS, Tc, TN, TN2)),
                      d4_2(treg[0], treg[1], treg[2], treg[3], treg[4]));
          }
          if constexpr (DM) {
#pragma unroll
            for (int d = 0; d < 3; d++) dmv[d] = dmom(d, f4);
          }
        } else {
          const DiffCol &Q0 = D.dcol[own], &Q1 = D.dcol[own + 1];
          const int offz[4] = {-2, -1, 1, 2};
          if constexpr (DS) {
            bool fx0[4], fx1[4], fy0[4], fy1[4], fz0[4], fz1[4];
#pragma unroll
            for (int a = 0; a < 4; a++) {
              fx0[a] = fluid_at(k, Q0.cx[a], Q0.ctop);
              fx1[a] = fluid_at(k, Q1.cx[a], Q1.ctop);
              fy0[a] = fluid_at(k, Q0.cy[a], Q0.ctop);
              fy1[a] = fluid_at(k, Q1.cy[a], Q1.ctop);
              fz0[a] = fluid_at(k + offz[a], Q0.c0, Q0.ctop);
              fz1[a] = fluid_at(k + offz[a], Q1.c0, Q1.ctop);
            }
            const float *Tk = S.to;
            const float2 Tm2 = ld2(Tk + c - 2), Tc = ld2(Tk + c), Tp2 = ld2(Tk + c + 2);
            const float2 Tl = odd2(Tm2, Tc), Tr = odd2(Tc, Tp2);
            const float2 TS2 = ld2(Tk + c - 2 * HX), TS = ld2(Tk + c - HX), TN = ld2(Tk + c + HX),
                         TN2 = ld2(Tk + c + 2 * HX);
            dd = add2(add2(dax2(Tm2, Tl, Tc, Tr, Tp2, true, fx0, fx1), dax2(TS2, TS, Tc, TN, TN2, true, fy0, fy1)),
                      dax2(treg[0], treg[1], treg[2], treg[3], treg[4], true, fz0, fz1));
          }
          if constexpr (DM) {
            bool gx0[4], gx1[4], gy0[4], gy1[4], gz0[4], gz1[4];
#pragma unroll
            for (int a = 0; a < 4; a++) {
              gx0[a] = fluid_at(k, Q0.vx[a], Q0.vtop);
              gx1[a] = fluid_at(k, Q1.vx[a], Q1.vtop);
              gy0[a] = fluid_at(k, Q0.vy[a], Q0.vtop);
              gy1[a] = fluid_at(k, Q1.vy[a], Q1.vtop);
              gz0[a] = fluid_at(k + offz[a], Q0.v0, Q0.vtop);
              gz1[a] = fluid_at(k + offz[a], Q1.v0, Q1.vtop);
            }
            auto fw = [&](int axis, float2 a, float2 b, float2 c_, float2 d, float2 e) {
              return axis == 0 ? dax2(a, b, c_, d, e, false, gx0, gx1)
                               : axis == 1 ? dax2(a, b, c_, d, e, false, gy0, gy1) : dax2(a, b, c_, d, e, false, gz0, gz1);
            };
#pragma unroll
            for (int d = 0; d < 3; d++) dmv[d] = dmom(d, fw);
          }
        }

        float2 rN_ = bc2(0.0f), pN_ = bc2(0.0f), rF_ = bc2(0.0f), pF_ = bc2(0.0f);
        if constexpr (DS) {
          // ---- scalar update: rho', p' (Sec 2.4), leapfrog and filter
          const float2 Dth = mul2(bc2(-kdif), dd);
          const float2 rC_ = ld2(S.cr[ck] + c), pC_ = ld2(S.cp[ck] + c), pO_ = ld2(S.op[ok4] + c);
          const float2 dtv = bc2(dt2);
          rN_ = sub2(rO_, mul2(dtv, mul2(RM, bc2(v0inv))));
          pN_ = sub2(pO_, mul2(mul2(mul2(dtv, bc2(Cp)), ek0.exner(E, pC_)), sub2(mul2(RH, bc2(v0inv)), Dth)));
          if (k < kug0) {
            rN_.x = 0.0f;
            pN_.x = 0.0f;
          }
          if (k < kug1) {
            rN_.y = 0.0f;
            pN_.y = 0.0f;
          }
          rF_ = fma2(bc2(nu), add2(sub2(rN_, mul2(bc2(2.0f), rC_)), rO_), rC_);
          pF_ = fma2(bc2(nu), add2(sub2(pN_, mul2(bc2(2.0f), pC_)), pO_), pC_);
          if (k < kug0) {
            rF_.x = 0.0f;
            pF_.x = 0.0f;
          }
          if (k < kug1) {
            rF_.y = 0.0f;
            pF_.y = 0.0f;
          }
        }

        if constexpr (DM) {
          // ---- velocity cells centred on the corners (c, c+1): Eqs. momentum_u_d .. w_d
          // vertical pair sums of the four cell columns around each corner: the
          // south-west columns (c-HX-1, c-HX) and west (c-1, c) as odd pairs
          const float2 Rmc = ld2(Rm + c), RmS = ld2(Rm + c - HX), RmS2 = ld2(Rm + c - HX - 2), Rm2 = ld2(Rm + c - 2);
          const float2 RS2 = ld2(R0 + c - HX - 2);
          const float2 cS = RS, cSW = odd2(RS2, RS), cW = odd2(Rl, Rc);
          const float2 mS = RmS, mSW = odd2(RmS2, RmS), mW = odd2(Rm2, Rmc);
          const float2 v00 = add2(mSW, cSW), v10 = add2(mS, cS), v01 = add2(mW, cW), v11 = add2(Rmc, Rc);
          const float2 q = bc2(0.25f);
          const float2 rE = mul2(add2(v10, v11), q), rW = mul2(add2(v00, v01), q);
          const float2 rNn = mul2(add2(v01, v11), q), rS = mul2(add2(v00, v10), q);
          const float2 rT = mul2(add2(add2(cSW, cS), add2(cW, Rc)), q);
          const float2 rB = mul2(add2(add2(mSW, mS), add2(mW, Rmc)), q);
          // corner velocities: this pair (c, c+1), its x-neighbours (c-1, c) and
          // (c+1, c+2), y-neighbours and the planes above and below
          const float *uxm = S.uu[ukm][0], *uym = S.uu[ukm][1], *uzm = S.uu[ukm][2];
          float2 u0[3], uE[3], uW[3], uN[3], uS[3], uT[3], uB[3];
          {
            const float *uk3[3] = {ux0, uy0, uz0}, *up3[3] = {uxp, uyp, uzp}, *um3[3] = {uxm, uym, uzm};
    #pragma unroll
            for (int d = 0; d < 3; d++) {
              const float2 a = ld2(uk3[d] + c - 2), b = ld2(uk3[d] + c), e = ld2(uk3[d] + c + 2);
              u0[d] = b;
              uW[d] = odd2(a, b);
              uE[d] = odd2(b, e);
              uN[d] = ld2(uk3[d] + c + HX);
              uS[d] = ld2(uk3[d] + c - HX);
              uT[d] = ld2(up3[d] + c);
              uB[d] = ld2(um3[d] + c);
            }
          }
          const float2 gE = mul2(mul2(rE, add2(u0[0], uE[0])), bc2(hSx)), gW = mul2(mul2(rW, add2(uW[0], u0[0])), bc2(hSx));
          const float2 gN = mul2(mul2(rNn, add2(u0[1], uN[1])), bc2(hSy)), gS = mul2(mul2(rS, add2(uS[1], u0[1])), bc2(hSy));
          const float2 gT = mul2(mul2(rT, add2(u0[2], uT[2])), bc2(hSz)), gB = mul2(mul2(rB, add2(uB[2], u0[2])), bc2(hSz));
          const float2 gsum = add2(add2(sub2(gE, gW), sub2(gN, gS)), sub2(gT, gB));
          // pressure sums and the buoyancy mean (rho' of the eight cells)
          const float *P0 = S.cp[ck], *Pm = S.cp[ckm];
          const float2 P0c = ld2(P0 + c), P0S = ld2(P0 + c - HX), P0S2 = ld2(P0 + c - HX - 2), P02 = ld2(P0 + c - 2);
          const float2 Pmc = ld2(Pm + c), PmS = ld2(Pm + c - HX), PmS2 = ld2(Pm + c - HX - 2), Pm2 = ld2(Pm + c - 2);
          const float2 pcSW = odd2(P0S2, P0S), pcW = odd2(P02, P0c), pmSW = odd2(PmS2, PmS), pmW = odd2(Pm2, Pmc);
          const float2 w00 = add2(pmSW, pcSW), w10 = add2(PmS, P0S), w01 = add2(pmW, pcW), w11 = add2(Pmc, P0c);
          const float2 pE = add2(w10, w11), pW = add2(w00, w01), pNn = add2(w01, w11), pS = add2(w00, w10);
          const float2 pT = add2(add2(pcSW, P0S), add2(pcW, P0c));
          const float2 pB = add2(add2(pmSW, PmS), add2(pmW, Pmc));
          const float *Q0p = S.cr[ck], *Qmp = S.cr[ckm];
          const float2 Q0c = ld2(Q0p + c), Q0S = ld2(Q0p + c - HX), Q0S2 = ld2(Q0p + c - HX - 2), Q02 = ld2(Q0p + c - 2);
          const float2 Qmc = ld2(Qmp + c), QmS = ld2(Qmp + c - HX), QmS2 = ld2(Qmp + c - HX - 2), Qm2 = ld2(Qmp + c - 2);
          const float2 r8 = add2(add2(add2(odd2(Q0S2, Q0S), Q0S), add2(odd2(Q02, Q0c), Q0c)),
                                 add2(add2(odd2(QmS2, QmS), QmS), add2(odd2(Qm2, Qmc), Qmc)));
          const float2 pg[3] = {mul2(sub2(pE, pW), bc2(qdx)), mul2(sub2(pNn, pS), bc2(qdy)), mul2(sub2(pT, pB), bc2(qdz))};
          const float2 mcur[3] = {ld2(S.cm[sk][0] + c), ld2(S.cm[sk][1] + c), ld2(S.cm[sk][2] + c)};
          float2 mnew[3], mflt[3];
    #pragma unroll
          for (int d = 0; d < 3; d++) {
            const float2 adv =
                fma2(u0[d], gsum,
                     add2(add2(sub2(mul2(gE, uE[d]), mul2(gW, uW[d])), sub2(mul2(gN, uN[d]), mul2(gS, uS[d]))),
                          sub2(mul2(gT, uT[d]), mul2(gB, uB[d]))));
            float2 tend = sub2(mul2(adv, bc2(-v0inv)), pg[d]);
            if (d == 2) tend = sub2(tend, mul2(bc2(g * 0.125f), r8));
            const float2 ref0 = bc2(d == 0 ? rbc[2] : 0.0f);
            const float2 mold = mo(2, d);
            tend = sub2(tend, fma2(bc2(kdif), dmv[d], mul2(bc2(tk), sub2(mold, ref0))));
            mnew[d] = fma2(bc2(dt2), tend, mold);
            mflt[d] = fma2(bc2(nu), add2(sub2(mnew[d], mul2(bc2(2.0f), mcur[d])), mold), mcur[d]);
          }
          {
            const float2 chk = add2(add2(mnew[0], mnew[1]), mnew[2]);
            const float cx = q0 ? chk.x : 0.0f, cy = q1 ? chk.y : 0.0f;
            if (!isfinite(cx) || !isfinite(cy)) wflag |= WATCH_NONFINITE;
            const float2 cou = fma2(make_float2(fabsf(u0[0].x), fabsf(u0[0].y)), bc2(cfx),
                                    fma2(make_float2(fabsf(u0[1].x), fabsf(u0[1].y)), bc2(cfy),
                                         mul2(make_float2(fabsf(u0[2].x), fabsf(u0[2].y)), bc2(cfz))));
            if ((a0 && cou.x > 1.0f) || (a1 && cou.y > 1.0f)) wflag |= WATCH_COURANT;
          }
          // stores after every shared-memory read of the plane: both corners as
          // one 8-byte store where both are computed
#pragma unroll
          for (int d = 0; d < 3; d++) {
            if (q0 && q1) {
              st2(mN[d] + o, mnew[d]);
              st2(mF[d] + o, mflt[d]);
            } else if (q0) {
              mN[d][o] = mnew[d].x;
              mF[d][o] = mflt[d].x;
            } else if (q1) {
              mN[d][o + 1] = mnew[d].y;
              mF[d][o + 1] = mflt[d].y;
            }
          }
        }
        if constexpr (DS) {
          const float2 chk = add2(rN_, pN_);
          const float cx = a0 ? chk.x : 0.0f, cy = a1 ? chk.y : 0.0f;
          if (!isfinite(cx) || !isfinite(cy)) wflag |= WATCH_NONFINITE;
          if (a0 && a1) {
            st2(rpN + o, rN_);
            st2(ppN + o, pN_);
            st2(rpF + o, rF_);
            st2(ppF + o, pF_);
          } else if (a0) {
            rpN[o] = rN_.x;
            ppN[o] = pN_.x;
            rpF[o] = rF_.x;
            ppF[o] = pF_.x;
          } else if (a1) {
            rpN[o + 1] = rN_.y;
            ppN[o + 1] = pN_.y;
            rpF[o + 1] = rF_.y;
            ppF[o + 1] = pF_.y;
          }
        }
      }
#pragma unroll
      for (int a = 0; a < 4; a++) {
        if constexpr (DS) treg[a] = treg[a + 1];
        if constexpr (DM) {
          if (NR == 1 || a == 0) {
            mreg[a][0] = mreg[a + 1][0];
            mreg[a][1] = mreg[a + 1][1];
            mreg[a][2] = mreg[a + 1][2];
          } else if (a == 1) {
            const int a4 = s4(k);
            mreg[1][0] = ld2(S.om[a4][0] + c);
            mreg[1][1] = ld2(S.om[a4][1] + c);
            mreg[1][2] = ld2(S.om[a4][2] + c);
          }
        }
      }
    }
    return wflag;
  };
  unsigned wflag;
  if constexpr (NR == 1)
    wflag = march(RoleTag<true>{}, RoleTag<true>{});
  else if (role == 0)
    wflag = march(RoleTag<true>{}, RoleTag<false>{});
  else
    wflag = march(RoleTag<false>{}, RoleTag<true>{});
  await_groups<0>();
  if (aborted()) {
    // a plane's copies did not arrive: wait (bounded) for every copy in
    // flight before the block's shared memory is given up
    if (tid == 0)
      for (int kk = max(k0 - 2, issued - (PAIR_NBAR - 1)); kk <= issued; kk++) {
        const int u = kk - (k0 - 2);
        mbar_wait(&S.bar[u & (PAIR_NBAR - 1)], (unsigned)(u / PAIR_NBAR) & 1u, PAIR_DRAIN_NS);
      }
    wflag |= WATCH_TIMEOUT;
  }
  wflag = __reduce_or_sync(0xffffffffu, wflag);
  if (wflag && (tid & 31) == 0 && watch) atomicOr(watch, wflag);
}
