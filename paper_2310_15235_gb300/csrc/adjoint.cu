// Adjoint of the TREVR2 reverse ray trace: dLoss/dkappa and dLoss/dL for a
// loss whose gradient with respect to J is given.
//
// The forward map, per receiver i and band b (Sec. 2.5, Sec. 2.6):
//   J_ib = F_ib sum_src L_src,b w(r) exp(-tau_src,b),
//   tau_src,b = (r/s) tau_k,b(s),  tau_k,b(s) = sum_seg alpha_seg,b |seg n [0, s]|,
// F = 1/size^2 (times Eq. taucorr's factor with THICK), alpha of accepted
// internal cells from the transmission average of their halves
// (Eq. transmissionavg), bucket alpha = sum kappa m / V_box at leaves, cell
// luminosities summed from elements and cells placed at their centre of
// luminosity.  The discrete choices (the cut, beams, tree) are held fixed;
// the traversals are recomputed, nothing from the forward is stored.
//
// The adjoint runs in four steps:
//  1. walk (one warp per receiver, as the forward): the sources are found
//     and binned exactly as in the forward.  Each lane then walks its beam
//     twice.  Front to back it recomputes tau at every source and adds
//       dLoss/dL_src,b  += gJ_ib F_ib w e^{-tau},
//       dLoss/dc_src    += sum_b c_b [ (w'/w) rhat - dtau_b/dc ]  (cells only),
//       dtau/dc = (r/s) alpha(s) n + (tau_k(s)/s) (rhat - (r/s) n),
//     with c_b = gJ_ib F_ib L_b w e^{-tau_b}, and keeps q_b = c_b r/s per
//     source, and records the beam's segments.  Back to front (over the
//     recorded segments, or walking the beam again far half first when it
//     had more than the record holds) it carries W_b = sum of q_b over the
//     sources beyond the current segment [t0, t1) and adds to the cell
//       dLoss/dalpha_b -= W_b (t1 - t0) + sum_{t0 <= s < t1} q_b (s - t0),
//     so every segment costs O(1) however many sources lie past it.
//  2. tables, top down: dalpha_parent/dalpha_half from Eq. transmissionavg,
//       dalpha/da1 = [w1 e^{-d a1} + w12/2 e^{-d(a1+a2)/2}] / T,
//     into the halves (direction by direction for internal halves, summed
//     over directions for isotropic leaves).
//  3. elements: dLoss/dkappa_e = dLoss/dalpha_leaf m_e / V_leaf (+ the
//     receiver's own Eq. taucorr term); dLoss/dL_e sums, over the cells that
//     hold e, the cell's luminosity gradient plus its centre gradient times
//     dc/dL_e = (x_e - c)/L_tot, and adds e's own term as a point source.
#include <cfloat>
#include <cmath>
#include <cstdint>
#include <cstring>

#include "walk.cuh"

namespace trevr2 {

namespace {

struct AdjArgs {
  WalkArgs w;
  const float* gJ;   // [A][nbsel] upstream gradient
  float* g_atab;     // [n_internal][P][NBP] dLoss/dalpha of accepted internal cells
  float* g_aleaf;    // [n][NBP] dLoss/dalpha_leaf
  float* g_Lnode;    // [n][NBP] dLoss/dL of cells as point sources
  float4* g_c;       // [n] dLoss/d(centre of luminosity), normalised units (w unused)
  float* g_Lelem;    // [N][NBP] dLoss/dL of elements as point sources (sorted order)
  float* g_thick;    // [N][NBP] Eq. taucorr's dLoss/dkappa (sorted order)
  float* T;          // [warps][M][NBP] tau_k(s) of every staged source
  float* Q;          // [warps][M][NBP] alpha at s, then q_b = c_b r/s
  float4* seg;       // [warps][seg_cap][32] per lane: segment target, t0, t1
  int seg_cap;       // segments recorded per lane and pass (0: always walk again)
};

// Segments recorded front to back, replayed back to front: per lane and pass.
constexpr int kSegCap = 128;
constexpr int kAdjWarps = 8;  // warps per block of the adjoint walk
// Blocks per SM it is compiled for (80 registers): measured faster than 2
// blocks at 120 registers and than 7 blocks of 4 warps at 72.
constexpr int kAdjBlocksPerSM = 3;
// Beam record in shared memory: recording lane (5 bits), first record
// (13 bits), count (14 bits); kBeamRewalk marks a beam whose records did not fit.
constexpr uint32_t kBeamRewalk = 0x3fffu;

template <int NBP>
__device__ __forceinline__ void add_bands(float* __restrict__ dst, const float* v) {
  if constexpr (NBP == 4) {
    atomicAdd(reinterpret_cast<float4*>(dst), make_float4(v[0], v[1], v[2], v[3]));
  } else if constexpr (NBP == 2) {
    atomicAdd(reinterpret_cast<float2*>(dst), make_float2(v[0], v[1]));
  } else {
    atomicAdd(dst, v[0]);
  }
}

// The absorption gradient of one segment [t0, t1) of a beam (back to front):
// W holds sum q over the sources beyond t1, p2 the nearest source not yet
// passed.
template <int NBP>
__device__ __forceinline__ void segment_gradient(float* __restrict__ dst, float t0, float t1,
                                                 const SrcEntry* V, const float* Q, int start,
                                                 int& p2, float* W) {
  while (p2 >= start && !(V[p2].s < t1)) {
    const BandVec<NBP> qv = load_bands<NBP>(Q + int64_t(p2) * NBP);
#pragma unroll
    for (int b = 0; b < NBP; ++b) W[b] += qv.v[b];
    --p2;
  }
  float gin[NBP], win[NBP];
#pragma unroll
  for (int b = 0; b < NBP; ++b) gin[b] = win[b] = 0.0f;
  while (p2 >= start && V[p2].s >= t0) {
    const float ds = V[p2].s - t0;
    const BandVec<NBP> qv = load_bands<NBP>(Q + int64_t(p2) * NBP);
#pragma unroll
    for (int b = 0; b < NBP; ++b) {
      gin[b] += qv.v[b] * ds;
      win[b] += qv.v[b];
    }
    --p2;
  }
  float ga[NBP];
  bool any = false;
#pragma unroll
  for (int b = 0; b < NBP; ++b) {
    ga[b] = -(W[b] * (t1 - t0) + gin[b]);
    any |= ga[b] != 0.0f;
    W[b] += win[b];
  }
  if (any) add_bands<NBP>(dst, ga);
}

// d ln g / dr of Eq. intint's kernel g(r) = G(x)/h^2, x = r/(0.4886 h).
// G(x) = 1 - sum_m x^{2m}/(4m^2-1) for x < 1 and sum_m x^{-2m}/(4m^2-1) for
// x > 1 (the series of the closed form); G' has a log singularity at x = 1,
// where 0 is returned (a set of measure zero).
__device__ float soft_dlog(float r, float h) {
  const float ch = 0.48860251190292f * h;
  const float x = r / ch;
  if (x == 1.0f) return 0.0f;
  float G, dG;
  if (x < 0.5f) {
    const float x2 = x * x;
    float xm = 1.0f, s = 0.0f, ds = 0.0f;  // xm = x^{2m-2}
    for (int m = 1; m < 40; ++m) {
      const float c = 1.0f / float(4 * m * m - 1);
      ds += 2.0f * m * xm * x * c;
      xm *= x2;
      s += xm * c;
      if (xm < 1e-9f) break;
    }
    G = 1.0f - s;
    dG = -ds;
  } else if (x <= 2.0f) {
    const float xm = x - 1.0f, xp = x + 1.0f;
    const float l = logf((xm * xm) / (xp * xp));
    G = 0.5f * (1.0f + (x * x - 1.0f) / (4.0f * x) * l);
    dG = 0.5f * (0.25f * (1.0f + 1.0f / (x * x)) * l + 1.0f / x);
  } else {
    const float ix2 = 1.0f / (x * x);
    float xm = 1.0f, s = 0.0f, ds = 0.0f;
    for (int m = 1; m < 64; ++m) {
      xm *= ix2;
      const float term = xm / float(4 * m * m - 1);
      s += term;
      ds += 2.0f * m * term;
      if (term < 1e-9f * s) break;
    }
    G = s;
    dG = -ds / x;
  }
  return dG / (G * ch);
}

// Eq. taucorr's factor f(tau) = (1 - e^{-tau})/tau and its derivative.
__device__ __forceinline__ double thick_factor(double tau) {
  return tau > 0.0 ? -expm1(-tau) / tau : 1.0;
}
__device__ __forceinline__ double thick_factor_deriv(double tau) {
  if (tau < 1e-3) return -0.5 + tau * (1.0 / 3.0 - tau * (0.125 - tau / 30.0));
  return (exp(-tau) * (1.0 + tau) - 1.0) / (tau * tau);
}

// Chord of beam (x, n) with the box of node nd, clipped to [0, tmax]; tx is
// the exit before the clip at tmax.
__device__ __forceinline__ bool beam_chord(const NodeW& nd, const float xv[3], const float n[3],
                                           const float inv[3], float tmax, float& t0, float& t1,
                                           float& tx) {
  const float3 e = node_ext(nd.meta);
  const float ext[3] = {e.x, e.y, e.z};
  t0 = 0.0f;
  tx = INFINITY;
  bool hit = true;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const float lo = nd.lo[c], hi = lo + ext[c];
    if (n[c] == 0.0f) {
      hit &= (lo <= xv[c]) && (xv[c] < hi);  // half-open box for a grazing beam
    } else {
      const float ta = (lo - xv[c]) * inv[c], tb = (hi - xv[c]) * inv[c];
      t0 = fmaxf(t0, fminf(ta, tb));
      tx = fminf(tx, fmaxf(ta, tb));
    }
  }
  t1 = fminf(tmax, tx);
  return hit && (t0 < t1);
}

// Stage 1, lanes take beams with sources: each walks its beam front to back
// (near half first), records tau_k(s) and the absorption at s of every
// source and the beam's absorbing segments.
template <int NBP>
__device__ void adjoint_stage1(const AdjArgs& g, float3 x, int si, int lane, int* lstk,
                               const SrcEntry* V, float* T, float* Q, float4* S, const int* off,
                               const int* order, int nbeams, uint32_t* binfo, int* next_beam) {
  const WalkArgs& a = g.w;
  const float xv[3] = {x.x, x.y, x.z};
  BandVec<NBP> zero;
#pragma unroll
  for (int b = 0; b < NBP; ++b) zero.v[b] = 0.0f;
  int nrec = 0;
  for (int idx = lane; idx < nbeams; idx = atomicAdd(next_beam, 1)) {
    const int k = order[idx];
    const int start = k ? off[k - 1] : 0;
    const int end = off[k];
    const float smax = V[end - 1].s;
    const float4 dn = a.dirs[k];
    const int pair = __float_as_int(dn.w);
    const float n[3] = {dn.x, dn.y, dn.z};
    float inv[3], nx[3];
    bool up[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      inv[c] = n[c] != 0.0f ? 1.0f / n[c] : 0.0f;
      nx[c] = xv[c] * inv[c];
      up[c] = n[c] > 0.0f;
    }
    float tau[NBP];
#pragma unroll
    for (int b = 0; b < NBP; ++b) tau[b] = 0.0f;
    // the last absorbing segment: its start, unclipped exit and alpha (the
    // farthest sources lie in it when it was clipped at smax)
    float seg_t0 = 0.0f, seg_x = 0.0f;
    BandVec<NBP> seg_al = zero;
    const int first = nrec;
    int ptr = start;
    float s_next = V[ptr].s;
    // stack entries carry the time the beam enters the cell (a crossed half's
    // entry time is exactly its own slab entry time), so a pop only needs the
    // exit time; halves are pushed only when crossed and absorbing
    int2* st2 = reinterpret_cast<int2*>(lstk);
    int sp = 0;
    {
      const NodeW root = a.nodes[0];
      float t0, t1;
      if ((root.meta & kMetaHasAlpha) && beam_chord_fx(root, xv, n, inv, nx, smax, t0, t1))
        st2[sp++] = make_int2(0, __float_as_int(t0));
    }
    while (sp > 0 && ptr < end) {
      const int2 en = st2[--sp];
      const int q = en.x;
      const float t0 = __int_as_float(en.y);
      const NodeW nd = a.nodes[q];
      float tx = INFINITY;
      {
        const float3 e3 = node_ext(nd.meta);
        const float ext3[3] = {e3.x, e3.y, e3.z};
#pragma unroll
        for (int c = 0; c < 3; ++c)
          if (n[c] != 0.0f)
            tx = fminf(tx, fmaf(up[c] ? nd.lo[c] + ext3[c] : nd.lo[c], inv[c], -nx[c]));
      }
      const float t1 = fminf(smax, tx);
      if (!(nd.meta & kMetaLeaf) && cell_opens(a, q, nd, x, si)) {
        bool lower_first, lower_hit, upper_hit;
        float lt0, lt1, ut0, ut1;
        crossed_halves_fx(nd, xv, n, inv, nx, node_ext(nd.meta).z, t0, t1, lower_first, lower_hit,
                          upper_hit, lt0, lt1, ut0, ut1);
        const bool near_hit = lower_first ? lower_hit : upper_hit;
        const bool far_hit = lower_first ? upper_hit : lower_hit;
        if (far_hit)
          st2[sp++] = make_int2(lower_first ? nd.child + 1 : nd.child,
                                __float_as_int(lower_first ? ut0 : lt0));
        if (near_hit)
          st2[sp++] = make_int2(lower_first ? nd.child : nd.child + 1,
                                __float_as_int(lower_first ? lt0 : ut0));
        continue;
      }
      const BandVec<NBP> al =
          (nd.meta & kMetaLeaf) ? load_bands<NBP>(a.alpha_leaf + int64_t(q) * NBP)
                                : load_bands<NBP>(a.alpha_tab + (int64_t(nd.aux) * a.P + pair) * NBP);
      if (nrec < g.seg_cap) {
        const int dst = (nd.meta & kMetaLeaf) ? -(q + 1) : nd.aux * a.P + pair;
        S[nrec * 32 + lane] = make_float4(__int_as_float(dst), t0, t1, 0.0f);
      }
      ++nrec;
      while (s_next < t1) {
        const float ds = fmaxf(0.0f, s_next - t0);
        BandVec<NBP> tk;
#pragma unroll
        for (int b = 0; b < NBP; ++b) tk.v[b] = tau[b] + al.v[b] * ds;
        store_bands<NBP>(T + int64_t(ptr) * NBP, tk);
        store_bands<NBP>(Q + int64_t(ptr) * NBP, s_next > t0 ? al : zero);
        ++ptr;
        s_next = ptr < end ? V[ptr].s : INFINITY;
      }
#pragma unroll
      for (int b = 0; b < NBP; ++b) tau[b] += al.v[b] * (t1 - t0);
      seg_t0 = t0;
      seg_x = tx;
      seg_al = al;
    }
    BandVec<NBP> tk;
#pragma unroll
    for (int b = 0; b < NBP; ++b) tk.v[b] = tau[b];
    for (; ptr < end; ++ptr) {
      const float s_ = V[ptr].s;
      store_bands<NBP>(T + int64_t(ptr) * NBP, tk);
      store_bands<NBP>(Q + int64_t(ptr) * NBP, s_ > seg_t0 && s_ < seg_x ? seg_al : zero);
    }
    const uint32_t count = nrec <= g.seg_cap ? uint32_t(nrec - first) : kBeamRewalk;
    binfo[k] = uint32_t(lane) | ((uint32_t(first) & 0x1fffu) << 5) | (count << 18);
  }
}

// Stage 2, all lanes over the staged sources: the term of J, dLoss/dL,
// dLoss/dc (cells only) and q_b = c_b r/s, with c_b = gJ_b F_b L_b w e^{-tau_b}
// and dtau/dc = (r/s) alpha(s) n + (tau_k(s)/s) (rhat - (r/s) n).
template <int NBP>
__device__ void adjoint_stage2(const AdjArgs& g, float3 x, int si, int lane, const SrcEntry* V,
                               const int* Up, const float* T, float* Q, int n, const float* gJf,
                               float* Js, float* Jc) {
  const WalkArgs& a = g.w;
  const float hr = a.hn[si];
  const bool soft = (a.flags & TREVR2_SOFT) != 0;
  for (int e = lane; e < n; e += 32) {
    const SrcEntry src = V[e];
    const bool elem = (src.ref & kRefElement) != 0;
    const int64_t idx = src.ref & 0x7fffffff;
    const BandVec<NBP> L = load_bands<NBP>(elem ? a.Lelem + idx * NBP : a.Lnode + idx * NBP);
    const BandVec<NBP> tk = load_bands<NBP>(T + int64_t(e) * NBP);
    const BandVec<NBP> as = load_bands<NBP>(Q + int64_t(e) * NBP);
    float dL[NBP], cb[NBP];
    BandVec<NBP> qv;
    bool any = false;
#pragma unroll
    for (int b = 0; b < NBP; ++b) {
      const float ex = expf(-tk.v[b] * src.rs);
      const float term = L.v[b] * src.w * ex;
      const float y = term - Jc[b];
      const float t = Js[b] + y;
      Jc[b] = (t - Js[b]) - y;
      Js[b] = t;
      dL[b] = gJf[b] * src.w * ex;
      any |= dL[b] != 0.0f;
      cb[b] = dL[b] * L.v[b];
      qv.v[b] = cb[b] * src.rs;
    }
    store_bands<NBP>(Q + int64_t(e) * NBP, qv);
    if (any) add_bands<NBP>(elem ? g.g_Lelem + idx * NBP : g.g_Lnode + idx * NBP, dL);
    if (!elem) {
      const float4 c = a.csrc[idx];
      const float vx = c.x - x.x, vy = c.y - x.y, vz = c.z - x.z;
      const float r = sqrtf(vx * vx + vy * vy + vz * vz);
      const float ir = 1.0f / r;
      const float dlg = soft ? soft_dlog(r, hr) : -2.0f * ir;
      const float4 nk = a.dirs[Up[e]];
      float fr = 0.0f, fn = 0.0f;  // coefficients of rhat and n
#pragma unroll
      for (int b = 0; b < NBP; ++b) {
        fr += cb[b] * (dlg - tk.v[b] / src.s);
        fn += cb[b] * src.rs * (tk.v[b] / src.s - as.v[b]);
      }
      if (fr != 0.0f || fn != 0.0f)
        atomicAdd(g.g_c + idx, make_float4(fr * vx * ir + fn * nk.x, fr * vy * ir + fn * nk.y,
                                           fr * vz * ir + fn * nk.z, 0.0f));
    }
  }
}

// Stage 3, lanes take beams again: the absorption gradient of every segment,
// back to front, from the records (or walking the beam again, far half
// first, when they did not fit).
template <int NBP>
__device__ void adjoint_stage3(const AdjArgs& g, float3 x, int si, int lane, int* lstk,
                               const SrcEntry* V, const float* Q, const float4* S, const int* off,
                               const int* order, int nbeams, const uint32_t* binfo,
                               int* next_beam) {
  const WalkArgs& a = g.w;
  const float xv[3] = {x.x, x.y, x.z};
  for (int idx = lane; idx < nbeams; idx = atomicAdd(next_beam, 1)) {
    const int k = order[idx];
    const int start = k ? off[k - 1] : 0;
    const int end = off[k];
    const uint32_t info = binfo[k];
    const uint32_t count = info >> 18;
    float W[NBP];
#pragma unroll
    for (int b = 0; b < NBP; ++b) W[b] = 0.0f;
    int p2 = end - 1;
    if (count != kBeamRewalk) {
      const int rl = int(info & 31u), first = int((info >> 5) & 0x1fffu);
      for (int j = int(count) - 1; j >= 0; --j) {
        const float4 r = S[(first + j) * 32 + rl];
        const int dst = __float_as_int(r.x);
        float* d = dst < 0 ? g.g_aleaf + int64_t(-dst - 1) * NBP : g.g_atab + int64_t(dst) * NBP;
        segment_gradient<NBP>(d, r.y, r.z, V, Q, start, p2, W);
      }
    } else {
      const float smax = V[end - 1].s;
      const float4 dn = a.dirs[k];
      const int pair = __float_as_int(dn.w);
      const float n[3] = {dn.x, dn.y, dn.z};
      float inv[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) inv[c] = n[c] != 0.0f ? 1.0f / n[c] : 0.0f;
      int sp = 1;
      lstk[0] = 0;
      while (sp > 0) {
        const int q = lstk[--sp];
        const NodeW nd = a.nodes[q];
        if (!(nd.meta & kMetaHasAlpha)) continue;
        float t0, t1, tx;
        if (!beam_chord(nd, xv, n, inv, smax, t0, t1, tx)) continue;
        if (!(nd.meta & kMetaLeaf) && cell_opens(a, q, nd, x, si)) {
          // far half on top of the stack
          bool lower_first, lower_hit, upper_hit;
          float lt0, lt1, ut0, ut1;
          crossed_halves(nd, xv, n, inv, t0, t1, lower_first, lower_hit, upper_hit, lt0, lt1,
                         ut0, ut1);
          const bool near_hit = lower_first ? lower_hit : upper_hit;
          const bool far_hit = lower_first ? upper_hit : lower_hit;
          if (near_hit) lstk[sp++] = lower_first ? nd.child : nd.child + 1;
          if (far_hit) lstk[sp++] = lower_first ? nd.child + 1 : nd.child;
          continue;
        }
        float* d = (nd.meta & kMetaLeaf) ? g.g_aleaf + int64_t(q) * NBP
                                         : g.g_atab + (int64_t(nd.aux) * a.P + pair) * NBP;
        segment_gradient<NBP>(d, t0, t1, V, Q, start, p2, W);
      }
    }
  }
}

template <int NBP>
__device__ __forceinline__ void adjoint_receiver(const AdjArgs& g, int64_t slot, int lane, int* stk,
                                                 int* off, uint32_t* binfo, int* next_beam,
                                                 int* lstk, SrcEntry* U, int* Up, SrcEntry* V,
                                                 float* T, float* Q, float4* S) {
  const WalkArgs& a = g.w;
  const int64_t io = a.active[slot];
  if (io < 0 || io >= a.N) {
    if (lane == 0) atomicOr(a.status, kStatusBadActive);
    return;
  }
  const int si = a.inv[io];
  // upstream gradient per band (bands may repeat in the selection)
  float gJb[NBP];
#pragma unroll
  for (int b = 0; b < NBP; ++b) gJb[b] = 0.0f;
  for (int j = 0; j < a.nbsel; ++j) {
    const float v = g.gJ[slot * a.nbsel + j];
#pragma unroll
    for (int b = 0; b < NBP; ++b)
      if (a.bsel[j] == b) gJb[b] += v;
  }
  const bool thick = (a.flags & TREVR2_THICK) != 0;
  const double h = double(a.hn[si]) * a.size;
  float gJf[NBP];
  bool any = false;
#pragma unroll
  for (int b = 0; b < NBP; ++b) {
    double f = a.inv_size2;
    if (thick) f *= thick_factor(double(a.km[int64_t(si) * NBP + b]) / (h * h));
    gJf[b] = float(double(gJb[b]) * f);
    any |= gJf[b] != 0.0f;
  }
  if (!any) return;
  const float4 xr = a.pos32[si];
  const float3 x = grazing_coords(a, si, make_float3(xr.x, xr.y, xr.z));
  float Js[NBP], Jc[NBP];
#pragma unroll
  for (int b = 0; b < NBP; ++b) Js[b] = Jc[b] = 0.0f;
  for (int lo = 0;; lo += a.M) {
    const int total = phase_sources(a, x, si, lane, stk, a.src_stack_cap, U, Up, lo);
    const int staged = min(total - lo, a.M);
    make_sources(a, x, si, lane, U, Up, staged);
    const int n = staged > 0 ? bin_sources(a, lane, U, Up, staged, V, off) : 0;
    if (n > 0) {
      // bin_sources leaves the beams in Up unsorted: put them in V's order
      for (int e = lane; e < a.npix; e += 32) {
        const int s0 = e ? off[e - 1] : 0, s1 = off[e];
        for (int j = s0; j < s1; ++j) Up[j] = e;
      }
      int* order = reinterpret_cast<int*>(binfo) + a.npix;
      const int nbeams = order_beams(a, lane, V, off, order, order + a.npix);
      if (lane == 0) *next_beam = 32;
      __syncwarp();
      adjoint_stage1<NBP>(g, x, si, lane, lstk, V, T, Q, S, off, order, nbeams, binfo, next_beam);
      __syncwarp();
      adjoint_stage2<NBP>(g, x, si, lane, V, Up, T, Q, n, gJf, Js, Jc);
      if (lane == 0) *next_beam = 32;
      __syncwarp();
      adjoint_stage3<NBP>(g, x, si, lane, lstk, V, Q, S, off, order, nbeams, binfo, next_beam);
      __syncwarp();
    }
    if (lo + a.M >= total) break;
  }
  if (!thick) return;
  // Eq. taucorr: J = F0 Jraw f(tau_i), tau_i = kappa_i m_i / h_i^2
#pragma unroll
  for (int b = 0; b < NBP; ++b) {
    double v = double(Js[b]) - double(Jc[b]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == b && b < a.nb && gJb[b] != 0.0f) {
      const double tau = double(a.km[int64_t(si) * NBP + b]) / (h * h);
      // dtau/dkappa = m / h^2; the element kernel applies the mass
      const double dk = double(gJb[b]) * a.inv_size2 * v * thick_factor_deriv(tau) / (h * h);
      atomicAdd(g.g_thick + int64_t(si) * NBP + b, float(dk));
    }
  }
}

// Shared memory of an adjoint block: per warp the stacks, the beam offsets,
// the beam records, the beam order and its 32 bucket counts, the next-beam
// counter and one pad int (an even count keeps the lane stacks' 8-byte
// entries aligned).
inline size_t adjoint_smem(int warps, int stack_ints, int npix) {
  return size_t(warps) * (stack_ints + 3 * npix + 34) * sizeof(int);
}

template <int NBP, int WARPS>
__global__ void __launch_bounds__(WARPS * 32, kAdjBlocksPerSM) k_walk_adjoint(const __grid_constant__ AdjArgs g) {
  extern __shared__ int smem[];
  const WalkArgs& a = g.w;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t gw = int64_t(blockIdx.x) * WARPS + wib;
  int* wsm = smem + wib * (a.stack_ints + 3 * a.npix + 34);  // even: 8-byte stack entries
  int* stk = wsm;
  int* off = wsm + a.stack_ints;
  uint32_t* binfo = reinterpret_cast<uint32_t*>(off + a.npix);
  int* next_beam = off + 3 * a.npix + 32;  // after the records, the order and its counts
  int* lstk = stk + lane * 2 * (a.max_depth + 2);
  SrcEntry* U = a.srcU + gw * a.M;
  int* Up = a.pixU + gw * a.M;
  SrcEntry* V = a.srcV + gw * a.M;
  float* T = g.T + gw * a.M * NBP;
  float* Q = g.Q + gw * a.M * NBP;
  float4* S = g.seg + gw * g.seg_cap * 32;
  for (;;) {
    unsigned long long slot = 0;
    if (lane == 0) slot = atomicAdd(a.counter, 1ull);
    slot = __shfl_sync(0xffffffffu, slot, 0);
    if (slot >= (unsigned long long)a.A) break;
    adjoint_receiver<NBP>(g, int64_t(slot), lane, stk, off, binfo, next_beam, lstk, U, Up, V, T, Q,
                          S);
  }
}

// Step 2: one depth of the tables' adjoint, parents before children.
template <int NBP>
__global__ void k_alpha_adjoint_level(int64_t lb, int64_t le, int P, int nb, bool linear,
                                      const NodeW* __restrict__ nodes,
                                      const int* __restrict__ int_index,
                                      const float* __restrict__ alpha_leaf,
                                      const TransGeo* __restrict__ geo,
                                      const float* __restrict__ tab, float* __restrict__ g_atab,
                                      float* __restrict__ g_aleaf) {
  const int64_t idx = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  const int64_t q = lb + idx / P;
  const int p = int(idx % P);
  if (q >= le) return;
  const NodeW nd = nodes[q];
  if (nd.child < 0) return;
  const int iq = int_index[q];
  const BandVec<NBP> G = load_bands<NBP>(g_atab + (int64_t(iq) * P + p) * NBP);
  bool any = false;
#pragma unroll
  for (int b = 0; b < NBP; ++b) any |= G.v[b] != 0.0f;
  if (!any) return;
  const int depth = int(nd.meta & kMetaDepthMask);
  const TransGeo gg = geo[(depth % 3) * P + p];
  const float d = ldexpf(gg.d_unit, -(depth / 3));
  const int c = nd.child;
  const int i1 = int_index[c], i2 = int_index[c + 1];
  const BandVec<NBP> a1 = i1 < 0 ? load_bands<NBP>(alpha_leaf + int64_t(c) * NBP)
                                 : load_bands<NBP>(tab + (int64_t(i1) * P + p) * NBP);
  const BandVec<NBP> a2 = i2 < 0 ? load_bands<NBP>(alpha_leaf + int64_t(c + 1) * NBP)
                                 : load_bands<NBP>(tab + (int64_t(i2) * P + p) * NBP);
#pragma unroll
  for (int b = 0; b < NBP; ++b) {
    if (b >= nb || G.v[b] == 0.0f) continue;
    // T = w1 e^{-x1} + w1 e^{-x2} + w12 e^{-(x1+x2)/2}; dalpha/da1 = (dT/dx1)/(-T)
    const float x1 = d * a1.v[b], x2 = d * a2.v[b], x12 = 0.5f * (x1 + x2);
    float m = INFINITY;
    if (gg.w1 > 0.0f) m = fminf(x1, x2);
    if (gg.w12 > 0.0f) m = fminf(m, x12);
    const float e1 = gg.w1 > 0.0f ? gg.w1 * expf(-(x1 - m)) : 0.0f;
    const float e2 = gg.w1 > 0.0f ? gg.w1 * expf(-(x2 - m)) : 0.0f;
    const float e12 = gg.w12 > 0.0f ? gg.w12 * expf(-(x12 - m)) : 0.0f;
    const float iS = 1.0f / (e1 + e2 + e12);
    // linear average: dalpha/dalpha_1 = dalpha/dalpha_2 = 1/2
    const float d1 = linear ? 0.5f * G.v[b] : G.v[b] * (e1 + 0.5f * e12) * iS;
    const float d2 = linear ? 0.5f * G.v[b] : G.v[b] * (e2 + 0.5f * e12) * iS;
    if (i1 < 0) atomicAdd(g_aleaf + int64_t(c) * NBP + b, d1);
    else g_atab[(int64_t(i1) * P + p) * NBP + b] += d1;
    if (i2 < 0) atomicAdd(g_aleaf + int64_t(c + 1) * NBP + b, d2);
    else g_atab[(int64_t(i2) * P + p) * NBP + b] += d2;
  }
}

__global__ void k_leaf_of(int64_t n, const int* __restrict__ child, const int* __restrict__ first,
                          const int* __restrict__ count, int* __restrict__ leaf_of) {
  const int64_t q = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (q >= n || child[q] >= 0) return;
  const int f = first[q], c = count[q];
  for (int e = f; e < f + c; ++e) leaf_of[e] = int(q);
}

// Step 3: per element (caller order), FP64 sums over the cells that hold it.
template <int NBP>
__global__ void k_grad_elements(int64_t N, int nb, double inv_size2, const int* __restrict__ inv,
                                const int* __restrict__ leaf_of, const int* __restrict__ parent,
                                const int* __restrict__ depth, const float* __restrict__ mass,
                                const double* __restrict__ pos64, const float4* __restrict__ csrc,
                                const double* __restrict__ c64, const float* __restrict__ g_aleaf,
                                const float* __restrict__ g_Lnode, const float4* __restrict__ g_c,
                                const float* __restrict__ g_Lelem, const float* __restrict__ g_thick,
                                float* __restrict__ g_kappa, float* __restrict__ g_lum) {
  const int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (e >= N) return;
  const int64_t si = inv[e];
  const int leaf = leaf_of[si];
  const double m = double(mass[si]);
  // alpha_leaf = sum kappa m / (V_leaf size^2), V_leaf = 2^-depth (normalised)
  const double dadk = ldexp(m, depth[leaf]) * inv_size2;
  double gl[NBP];
#pragma unroll
  for (int b = 0; b < NBP; ++b) gl[b] = double(g_Lelem[si * NBP + b]);
  const double x[3] = {pos64[3 * si], pos64[3 * si + 1], pos64[3 * si + 2]};
  for (int q = leaf; q >= 0; q = parent[q]) {
#pragma unroll
    for (int b = 0; b < NBP; ++b) gl[b] += double(g_Lnode[int64_t(q) * NBP + b]);
    const float Lt = csrc[q].w;
    if (Lt > 0.0f) {
      double dot = 0.0;
      const float4 gc = g_c[q];
      const double gcv[3] = {double(gc.x), double(gc.y), double(gc.z)};
      for (int a = 0; a < 3; ++a) dot += gcv[a] * (x[a] - c64[3 * int64_t(q) + a]);
      dot /= double(Lt);
#pragma unroll
      for (int b = 0; b < NBP; ++b) gl[b] += dot;
    }
  }
#pragma unroll
  for (int b = 0; b < NBP; ++b) {
    if (b >= nb) continue;
    const double gk = double(g_aleaf[int64_t(leaf) * NBP + b]) * dadk +
                      double(g_thick[si * NBP + b]) * m;
    g_kappa[e * nb + b] = float(gk);
    g_lum[e * nb + b] = float(gl[b]);
  }
}

template <int NBP>
const void* adjoint_kernel() {
  return reinterpret_cast<const void*>(&k_walk_adjoint<NBP, kAdjWarps>);
}

}  // namespace

}  // namespace trevr2

using namespace trevr2;

extern "C" int trevr2_J_backward(trevr2_tree* tree, const int64_t* active, int64_t A, int nside,
                                 float theta, const int* bands, int nbsel, uint32_t flags,
                                 const float* gJ, float* g_kappa, float* g_lum, void* stream) {
  clear_error();
  if (!tree) {
    set_error("trevr2_J_backward: tree is NULL");
    return TREVR2_EINVAL;
  }
  Tree* t = reinterpret_cast<Tree*>(tree);
  const int64_t N = t->N;
  if (A < 0 || (A > 0 && (!active || !gJ)) || (N > 0 && (!g_kappa || !g_lum))) {
    set_error("trevr2_J_backward: A < 0 or NULL active/gJ/g_kappa/g_lum");
    return TREVR2_EINVAL;
  }
  if (!valid_nside(nside)) {
    set_error("trevr2_J_backward: nside %d is not a power of two in [1, %d]", nside,
              TREVR2_MAX_NSIDE);
    return nside > TREVR2_MAX_NSIDE ? TREVR2_EUNSUPPORTED : TREVR2_EINVAL;
  }
  if (!(theta > 0.0f) || !std::isfinite(theta)) {
    set_error("trevr2_J_backward: theta must be positive and finite");
    return TREVR2_EINVAL;
  }
  if (flags & (TREVR2_BUCKET | TREVR2_PP | TREVR2_CSM)) {
    set_error("trevr2_J_backward: TREVR2_BUCKET, TREVR2_PP and TREVR2_CSM are trevr2_J flags "
              "only");
    return TREVR2_EUNSUPPORTED;
  }
  if (flags & ~(TREVR2_SOFT | TREVR2_THICK | TREVR2_LINEAR | TREVR2_ASYNC)) {
    set_error("trevr2_J_backward: unknown flags 0x%x", flags);
    return TREVR2_EINVAL;
  }
  int bsel[TREVR2_MAX_BANDS];
  if (bands) {
    if (nbsel < 1 || nbsel > TREVR2_MAX_BANDS) {
      set_error("trevr2_J_backward: nbsel must be in [1, %d]", TREVR2_MAX_BANDS);
      return TREVR2_EINVAL;
    }
    for (int j = 0; j < nbsel; ++j) {
      if (bands[j] < 0 || bands[j] >= t->nb) {
        set_error("trevr2_J_backward: band %d out of range [0, %d)", bands[j], t->nb);
        return TREVR2_EINVAL;
      }
      bsel[j] = bands[j];
    }
  } else {
    nbsel = t->nb;
    for (int j = 0; j < nbsel; ++j) bsel[j] = j;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  t->last_stream = st;
  Table* tb = nullptr;
  const bool linear = (flags & TREVR2_LINEAR) != 0;
  T2_CHECK(ensure_table(t, nside, st, &tb, linear));
  const int P = 6 * nside * nside;
  const int nbp = t->nbp;
  const int64_t n = t->n_nodes;

  // launch shape of the walk
  WalkArgs wa;
  fill_walk_args(t, tb, nside, theta, bsel, nbsel, flags & ~TREVR2_ASYNC, kSrcCapacity, &wa);
  wa.A = A;
  wa.active = active;
  const void* fn = nbp == 1 ? adjoint_kernel<1>() : nbp == 2 ? adjoint_kernel<2>() : adjoint_kernel<4>();
  const size_t smem = adjoint_smem(kAdjWarps, wa.stack_ints, wa.npix);
  int per_sm = 0, sms = 0;
  T2_CHECK(config_walk_kernel(fn, kAdjWarps, smem, &per_sm, &sms));
  int64_t blocks = int64_t(sms) * per_sm;
  blocks = std::max<int64_t>(1, std::min<int64_t>(blocks, (A + kAdjWarps - 1) / kAdjWarps));
  const size_t warps = size_t(blocks) * kAdjWarps;

  // one allocation: gradient buffers (zeroed), leaf map, walk buffers
  auto up = [](size_t b) { return (b + 255) & ~size_t(255); };
  const size_t b_atab = up(sizeof(float) * size_t(std::max<int64_t>(t->n_internal, 1)) * P * nbp);
  const size_t b_aleaf = up(sizeof(float) * size_t(n) * nbp);
  const size_t b_Lnode = b_aleaf;
  const size_t b_c = up(sizeof(float4) * size_t(n));
  const size_t b_Lelem = up(sizeof(float) * size_t(N) * nbp);
  const size_t b_thick = b_Lelem;
  const size_t zeroed = b_atab + b_aleaf + b_Lnode + b_c + b_Lelem + b_thick;
  const size_t b_leaf = up(sizeof(int) * size_t(std::max<int64_t>(N, 1)));
  const size_t b_Q = up(sizeof(float) * warps * wa.M * nbp);
  const size_t b_T = b_Q;
  // segment records address the table by a 32-bit row index
  const int seg_cap = int64_t(std::max<int64_t>(t->n_internal, 1)) * P < INT32_MAX ? kSegCap : 0;
  const size_t b_seg = up(sizeof(float4) * warps * size_t(seg_cap) * 32);
  const size_t b_walk = warps * size_t(wa.M) * (2 * sizeof(SrcEntry) + sizeof(int));
  char* base = nullptr;
  T2_CHECK(device_alloc(reinterpret_cast<void**>(&base),
                        zeroed + b_leaf + b_T + b_Q + b_seg + b_walk, st, "adjoint buffers"));
  AdjArgs g;
  std::memset(&g, 0, sizeof(g));
  g.w = wa;
  g.gJ = gJ;
  char* p = base;
  g.g_atab = reinterpret_cast<float*>(p); p += b_atab;
  g.g_aleaf = reinterpret_cast<float*>(p); p += b_aleaf;
  g.g_Lnode = reinterpret_cast<float*>(p); p += b_Lnode;
  g.g_c = reinterpret_cast<float4*>(p); p += b_c;
  g.g_Lelem = reinterpret_cast<float*>(p); p += b_Lelem;
  g.g_thick = reinterpret_cast<float*>(p); p += b_thick;
  int* leaf_of = reinterpret_cast<int*>(p); p += b_leaf;
  g.T = reinterpret_cast<float*>(p); p += b_T;
  g.Q = reinterpret_cast<float*>(p); p += b_Q;
  g.seg = reinterpret_cast<float4*>(p); p += b_seg;
  g.seg_cap = seg_cap;
  g.w.srcU = reinterpret_cast<SrcEntry*>(p);
  g.w.srcV = reinterpret_cast<SrcEntry*>(p + warps * wa.M * sizeof(SrcEntry));
  g.w.pixU = reinterpret_cast<int*>(p + 2 * warps * wa.M * sizeof(SrcEntry));
  int rc = TREVR2_OK;
  auto run = [&]() -> int {
    T2_CUDA(cudaMemsetAsync(base, 0, zeroed, st));
    if (A > 0) {
      T2_CUDA(cudaMemsetAsync(t->counter, 0, sizeof(unsigned long long), st));
      void* args[] = {&g};
      T2_CUDA(cudaLaunchKernel(fn, dim3(unsigned(blocks)), dim3(kAdjWarps * 32), args, smem, st));
      note_launch();
    }
    for (int d = 0; d < t->max_depth; ++d) {
      const int64_t lb = t->level_begin[d], le = t->level_begin[d + 1];
      const int64_t work = (le - lb) * P;
      if (work == 0) continue;
      const unsigned nblk = unsigned((work + 255) / 256);
      switch (nbp) {
        case 1: k_alpha_adjoint_level<1><<<nblk, 256, 0, st>>>(lb, le, P, t->nb, linear, t->nodes, t->int_index, t->alpha_leaf, tb->geo, tb->alpha, g.g_atab, g.g_aleaf); break;
        case 2: k_alpha_adjoint_level<2><<<nblk, 256, 0, st>>>(lb, le, P, t->nb, linear, t->nodes, t->int_index, t->alpha_leaf, tb->geo, tb->alpha, g.g_atab, g.g_aleaf); break;
        default: k_alpha_adjoint_level<4><<<nblk, 256, 0, st>>>(lb, le, P, t->nb, linear, t->nodes, t->int_index, t->alpha_leaf, tb->geo, tb->alpha, g.g_atab, g.g_aleaf); break;
      }
      note_launch();
    }
    if (N > 0) {
      const unsigned nb_n = unsigned((n + 255) / 256);
      k_leaf_of<<<nb_n, 256, 0, st>>>(n, t->child, t->first, t->count, leaf_of);
      note_launch();
      const unsigned nb_e = unsigned((N + 255) / 256);
      const double is2 = 1.0 / (t->size * t->size);
      switch (nbp) {
        case 1: k_grad_elements<1><<<nb_e, 256, 0, st>>>(N, t->nb, is2, t->inv, leaf_of, t->parent, t->depth, t->mass, t->pos64, t->csrc, t->c64, g.g_aleaf, g.g_Lnode, g.g_c, g.g_Lelem, g.g_thick, g_kappa, g_lum); break;
        case 2: k_grad_elements<2><<<nb_e, 256, 0, st>>>(N, t->nb, is2, t->inv, leaf_of, t->parent, t->depth, t->mass, t->pos64, t->csrc, t->c64, g.g_aleaf, g.g_Lnode, g.g_c, g.g_Lelem, g.g_thick, g_kappa, g_lum); break;
        default: k_grad_elements<4><<<nb_e, 256, 0, st>>>(N, t->nb, is2, t->inv, leaf_of, t->parent, t->depth, t->mass, t->pos64, t->csrc, t->c64, g.g_aleaf, g.g_Lnode, g.g_c, g.g_Lelem, g.g_thick, g_kappa, g_lum); break;
      }
      note_launch();
    }
    T2_CUDA(cudaGetLastError());
    return TREVR2_OK;
  };
  rc = run();
  cudaFreeAsync(base, st);
  if (rc != TREVR2_OK) return rc;
  if (flags & TREVR2_ASYNC) return TREVR2_OK;
  return read_status(t, st);
}
