// The TREVR2 reverse ray trace (Sec. 2.5) on the GPU: J per active receiver.
//
// One warp per receiver, persistent grid, receivers taken from a global
// counter.  Two phases per receiver:
//
//  S (sources, warp-cooperative): a depth-first cut of the luminous part of
//    the tree with the opening criterion B/d > theta (Sec. 2.5.2); each
//    accepted luminous cell is a point source at its centre of luminosity,
//    each opened leaf gives its luminous elements (never the receiver
//    itself, Sec. 2.1).  Every source is put in the one HEALPix beam that
//    holds its direction (Sec. 2.5.1) with its projected distance s, r/s and
//    the kernel g(r) = 1/(4 pi r^2) (or Eq. intint), then the sources are
//    bucketed by beam and each bucket sorted by s.
//  A (absorption, lane per beam): each lane walks its beam front to back
//    through the same cut (near half first, so cells come in increasing
//    distance), skipping cells without absorption and stopping at the
//    farthest source of the beam.  Accepted internal cells use their
//    transmission-averaged alpha for the beam's direction pair, leaves their
//    bucket alpha.  Sources are resolved in order as the beam passes them:
//    tau(s) = tau(t_in) + alpha (s - t_in), scaled by r/s (Sec. 2.5.1), and
//    J_b += L_b e^{-tau_b} g(r) with a compensated FP32 sum per lane.
//  The lane partial sums are reduced in FP64, times Eq. taucorr with THICK.
//
// Discrete decisions (open or not, which beam) are taken in FP32 and taken
// again in FP64 when the FP32 margin is inside a guard band that bounds the
// FP32 error, so they agree with an FP64 evaluation.  Sources beyond the
// capacity of one warp's buffers are handled in further passes.
#include <cfloat>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "walk.cuh"

namespace trevr2 {

// Complex source model (Sec. 2.7): a cell's source adds its own ray's optical
// depth towards the bucket (direction -n_k) to the beam's.
template <int NBP>
__device__ __forceinline__ void add_csm(const WalkArgs& a, int ref, int k, BandVec<NBP>& tk) {
  if (ref & kRefElement) return;
  const BandVec<NBP> c =
      load_bands<NBP>(a.csm_tau + (int64_t(ref) * a.npix + a.csm_anti[k]) * NBP);
#pragma unroll
  for (int b = 0; b < NBP; ++b) tk.v[b] += c.v[b];
}

// Box extents for phase A's stack pops, the same values as node_ext: the
// longest side 2^-floor(depth / 3) by depth in shared memory (256 bytes, so
// that the walk kernels keep their blocks per SM), the others halved on the
// axes already split at this depth.  x, y, z, and w = the split axis's extent
// (z's).  Every kernel that runs phase A fills the table before its first
// receiver.
__shared__ float g_ext_e[64];

__device__ __forceinline__ void init_ext_tab() {
  if (threadIdx.x < 64) g_ext_e[threadIdx.x] = __int_as_float((127 - int(threadIdx.x) / 3) << 23);
  __syncthreads();
}

__device__ __forceinline__ float4 ext_of(uint32_t meta) {
  const float e = g_ext_e[meta & kMetaDepthMask];
  const uint32_t r = (meta >> kMetaAxisShift) & 3u;
  return make_float4(r > 0u ? 0.5f * e : e, r > 1u ? 0.5f * e : e, e, e);
}

// Phase A: lanes take beams from the order above through a per-warp counter.
// Each beam first descends the receiver's ancestors (chain[0..], root to the
// receiver's leaf, in shared memory): they hold the receiver, so they open,
// and each one's chord is its parent's near-half interval; only their
// crossed far halves go on the stack.  The stack walk then takes the far
// halves, nearest first.  This visits the same cells in the same order as a
// walk from the root.
template <int NBP, bool kBucket = false, bool kPP = false, bool kCSM = false>
__device__ void phase_absorb(const WalkArgs& a, float3 x, int si, int lane, int* lstk,
                             const SrcEntry* V, float* T, const int* off, const int* order,
                             int nbeams, int* next_beam, const NodeW* chain, int leaf,
                             float rpp = 0.0f) {
  int idx = lane;
  for (;;) {
    if (idx >= nbeams) break;
    const int k = order[idx];
    int ptr = k ? off[k - 1] : 0;
    const int end = off[k];
    const float smax = V[end - 1].s;
    float s_next = V[ptr].s;  // the nearest source not yet passed
    float4 dn = a.dirs[k];
    if constexpr (kBucket) {  // the directed beam (Sec. 3.4.1) points at its target
      const double* o = origin64<true>(a, si);
      if (int(o[7]) == k) dn = make_float4(float(o[4]), float(o[5]), float(o[6]), dn.w);
    }
    const int pair = __float_as_int(dn.w);
    const float n[3] = {dn.x, dn.y, dn.z};
    float inv[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) inv[c] = n[c] != 0.0f ? 1.0f / n[c] : 0.0f;
    const float xv[3] = {x.x, x.y, x.z};
    // slab times are face * inv - nx, one FMA; nx = -inf on an axis with
    // n = 0 makes that axis's exit time +inf
    float nx[3], upf[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      nx[c] = n[c] != 0.0f ? xv[c] * inv[c] : -INFINITY;
      upf[c] = n[c] > 0.0f ? 1.0f : 0.0f;  // the exit face is lo + upf * ext
    }
    float tau[NBP];
#pragma unroll
    for (int b = 0; b < NBP; ++b) tau[b] = 0.0f;
    // a cell of the cut crossed on [t0, t1): sources inside it, then its tau
    auto segment = [&](int q, const NodeW& nd, float t0, float t1) {
      // with a p-p radius (Sec. 2.4), cells absorb only beyond it
      if constexpr (kPP) t0 = fmaxf(t0, rpp);
      if constexpr (kPP) t1 = fmaxf(t1, t0);
      const BandVec<NBP> al = (nd.meta & kMetaLeaf)
                                  ? load_bands<NBP>(a.alpha_leaf + int64_t(q) * NBP)
                                  : load_bands<NBP>(a.alpha_tab + (int64_t(nd.aux) * a.P + pair) * NBP);
      while (s_next < t1) {
        const float ds = fmaxf(0.0f, s_next - t0);
        BandVec<NBP> tk;
#pragma unroll
        for (int b = 0; b < NBP; ++b) tk.v[b] = tau[b] + al.v[b] * ds;
        if constexpr (kCSM) add_csm<NBP>(a, V[ptr].ref, k, tk);
        store_bands<NBP>(T + int64_t(ptr) * NBP, tk);
        ++ptr;
        s_next = ptr < end ? V[ptr].s : INFINITY;
      }
#pragma unroll
      for (int b = 0; b < NBP; ++b) tau[b] += al.v[b] * (t1 - t0);
    };
    // a pushed half carries the time the beam enters it (exactly its own slab
    // entry time), so a pop only needs the exit time
    int2* st2 = reinterpret_cast<int2*>(lstk);
    int sp = 0;
    {
      const NodeW root = chain[0];
      float t0, t1;
      bool go = (root.meta & kMetaHasAlpha) && beam_chord_fx(root, xv, n, inv, nx, smax, t0, t1);
      for (int kd = 0; go; ++kd) {
        const NodeW nd = chain[kd];
        if (nd.meta & kMetaLeaf) {
          segment(leaf, nd, t0, t1);
          break;
        }
        bool lower_first, lower_hit, upper_hit;
        float lt0, lt1, ut0, ut1;
        crossed_halves_fx<!kPP>(nd, xv, n, inv, nx, ext_of(nd.meta).w, t0, t1,
                          lower_first, lower_hit, upper_hit, lt0, lt1, ut0, ut1);
        const bool near_hit = lower_first ? lower_hit : upper_hit;
        const bool far_hit = lower_first ? upper_hit : lower_hit;
        if (far_hit)
          st2[sp++] = make_int2(lower_first ? nd.child + 1 : nd.child,
                                __float_as_int(lower_first ? ut0 : lt0));
        go = near_hit;
        t0 = lower_first ? lt0 : ut0;
        t1 = lower_first ? lt1 : ut1;
      }
    }
    while (sp > 0 && ptr < end) {
      const int2 e = st2[--sp];
      const int q = e.x;
      const float t0 = __int_as_float(e.y);
      const NodeW nd = a.nodes[q];
      const float4 et = ext_of(nd.meta);
      float t1 = smax;
      t1 = fminf(t1, fmaf(fmaf(et.x, upf[0], nd.lo[0]), inv[0], -nx[0]));
      t1 = fminf(t1, fmaf(fmaf(et.y, upf[1], nd.lo[1]), inv[1], -nx[1]));
      t1 = fminf(t1, fmaf(fmaf(et.z, upf[2], nd.lo[2]), inv[2], -nx[2]));
      if (!(nd.meta & kMetaLeaf) &&
          cell_opens_e<kBucket, kPP>(a, q, nd, make_float3(et.x, et.y, et.z), x, si, rpp)) {
        // the crossed halves, the near one (the side of the receiver) on top
        bool lower_first, lower_hit, upper_hit;
        float lt0, lt1, ut0, ut1;
        crossed_halves_fx<!kPP>(nd, xv, n, inv, nx, et.w, t0, t1, lower_first, lower_hit, upper_hit,
                          lt0, lt1, ut0, ut1);
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
      segment(q, nd, t0, t1);
    }
    // sources beyond the last absorbing cell of the beam
    BandVec<NBP> tk;
#pragma unroll
    for (int b = 0; b < NBP; ++b) tk.v[b] = tau[b];
    for (; ptr < end; ++ptr) {
      if constexpr (kCSM) {
        BandVec<NBP> tc = tk;
        add_csm<NBP>(a, V[ptr].ref, k, tc);
        store_bands<NBP>(T + int64_t(ptr) * NBP, tc);
      } else {
        store_bands<NBP>(T + int64_t(ptr) * NBP, tk);
      }
    }
    idx = atomicAdd(next_beam, 1);
  }
}

// The n staged sources, all lanes at once: J_b += L_b g(r) e^{-tau_k(s) r/s}
// with a compensated FP32 sum per lane.
template <int NBP>
__device__ __forceinline__ void eval_sources(const WalkArgs& a, int lane, const SrcEntry* V,
                                             const float* T, int n, float* Js, float* Jc) {
  for (int e = lane; e < n; e += 32) {
    const SrcEntry src = V[e];
    const float* Lp = (src.ref & kRefElement) ? a.Lelem + int64_t(src.ref & 0x7fffffff) * NBP
                                              : a.Lnode + int64_t(src.ref) * NBP;
    const BandVec<NBP> L = load_bands<NBP>(Lp);
    const BandVec<NBP> tk = load_bands<NBP>(T + int64_t(e) * NBP);
#pragma unroll
    for (int b = 0; b < NBP; ++b) {
      const float term = L.v[b] * src.w * expf(-tk.v[b] * src.rs);
      const float y = term - Jc[b];
      const float t = Js[b] + y;
      Jc[b] = (t - Js[b]) - y;
      Js[b] = t;
    }
  }
}

// J of one receiver (caller index io of the tree described by a) into
// Jrow[0, nbsel); the warp's shared stacks and buffers are passed in.
template <int NBP>
__device__ __forceinline__ void walk_receiver_si(const WalkArgs& a, int si, float* Jrow, int lane,
                                                 int* stk, int* off, int* next_beam, int* lstk,
                                                 SrcEntry* U, int* Up, SrcEntry* V, float* T) {
  const float4 xr = a.pos32[si];
  // the receiver in FP32, on the FP64 side of every box face
  const float3 x = grazing_coords(a, si, make_float3(xr.x, xr.y, xr.z));
  // the receiver's ancestors, root first
  NodeW* chain = reinterpret_cast<NodeW*>(off + 2 * a.npix + 36);
  const int leaf = build_chain(a.nodes, x, lane, chain);
  float Js[NBP], Jc[NBP];
#pragma unroll
  for (int b = 0; b < NBP; ++b) Js[b] = Jc[b] = 0.0f;
  for (int lo = 0;; lo += a.M) {
    const int total = phase_sources(a, x, si, lane, stk, a.src_stack_cap, U, Up, lo);
    const int staged = min(total - lo, a.M);
    make_sources(a, x, si, lane, U, Up, staged);
    const int n = staged > 0 ? bin_sources(a, lane, U, Up, staged, V, off) : 0;
    if (n > 0) {
      int* order = off + a.npix;
      const int nbeams = order_beams(a, lane, V, off, order, order + a.npix);
      if (lane == 0) *next_beam = 32;
      __syncwarp();
      phase_absorb<NBP>(a, x, si, lane, lstk, V, T, off, order, nbeams, next_beam, chain, leaf);
      __syncwarp();
      eval_sources<NBP>(a, lane, V, T, n, Js, Jc);
      __syncwarp();
    }
    if (lo + a.M >= total) break;
  }
  // FP64 reduction of the lane partial sums
  double Jd[NBP];
#pragma unroll
  for (int b = 0; b < NBP; ++b) {
    double v = double(Js[b]) - double(Jc[b]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    Jd[b] = v;
  }
  if (lane < a.nbsel) {
    const int b = a.bsel[lane];
    double v = 0.0;
#pragma unroll
    for (int c = 0; c < NBP; ++c)
      if (c == b) v = Jd[c];
    v *= a.inv_size2;
    if (a.flags & TREVR2_THICK) {
      // Eq. taucorr: <I> = I(0) (1 - e^{-tau})/tau, tau = kappa m / h^2
      const double h = double(a.hn[si]) * a.size;
      const double tau = double(a.km[int64_t(si) * NBP + b]) / (h * h);
      if (tau > 0.0) v *= -expm1(-tau) / tau;
    }
    Jrow[lane] = float(v);
  }
}

// The same for the receiver with caller index io (NaN row and a status bit
// for an index outside [0, N)).
template <int NBP>
__device__ __forceinline__ void walk_receiver(const WalkArgs& a, int64_t io, float* Jrow, int lane,
                                              int* stk, int* off, int* next_beam, int* lstk,
                                              SrcEntry* U, int* Up, SrcEntry* V, float* T) {
  if (io < 0 || io >= a.N) {
    if (lane == 0) atomicOr(a.status, kStatusBadActive);
    if (lane < a.nbsel) Jrow[lane] = __int_as_float(0x7fc00000);
    return;
  }
  walk_receiver_si<NBP>(a, a.inv[io], Jrow, lane, stk, off, next_beam, lstk, U, Up, V, T);
}

// One warp per receiver, receivers from a global counter.
template <int NBP, int WARPS>
__global__ void __launch_bounds__(WARPS * 32, kWalkWarpsPerSM / WARPS) k_walk(WalkArgs a) {
  init_ext_tab();
  extern __shared__ int smem[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t gw = int64_t(blockIdx.x) * WARPS + wib;
  int* wsm = smem + wib * (a.stack_ints + 2 * a.npix + 36 + 8 * (a.max_depth + 1));
  int* stk = wsm;
  int* off = wsm + a.stack_ints;
  int* next_beam = off + 2 * a.npix + 32;  // after the beam order and its counts
  int* lstk = stk + lane * 2 * (a.max_depth + 2);
  SrcEntry* U = a.srcU + gw * a.M;
  int* Up = a.pixU + gw * a.M;
  SrcEntry* V = a.srcV + gw * a.M;
  float* T = a.srcT + gw * a.M * 4;
  for (;;) {
    unsigned long long slot = 0;
    if (lane == 0) slot = atomicAdd(a.counter, 1ull);
    slot = __shfl_sync(0xffffffffu, slot, 0);
    if (slot >= (unsigned long long)a.A) break;
    const int64_t r = a.order ? int64_t(a.order[slot]) : int64_t(slot);
    walk_receiver<NBP>(a, a.active[r], a.J + r * a.nbsel, lane, stk, off, next_beam,
                       lstk, U, Up, V, T);
  }
}

// ---------------------------------------------------------------------------
// Per-bucket beams (TREVR2_BUCKET; Sec. 2 and Sec. 2.5.1).  One walk per
// bucket, the leaf that holds the receivers, from the centre of its box:
// the cut, each source's beam and projected distance s and the optical depth
// tau_k(s) are the bucket's.  Each receiver of the bucket then adds
// L g(r) e^{-tau_k(s) r/s} at its own distance r (its own h under
// TREVR2_SOFT, its own Eq. taucorr factor under TREVR2_THICK).  Receivers
// come in Morton order, so a bucket's receivers are adjacent; the warp that
// takes a bucket's first slot walks it, and other slots are passed over.

struct BucketArgs {
  const uint64_t* keys;  // [A] sorted element position of each slot (N: invalid)
  const int* leaf;       // [A] leaf of each slot (-1: invalid)
  uint32_t rflags;       // the receivers' flags (TREVR2_SOFT, TREVR2_THICK)
  // particle-particle absorption (TREVR2_PP, Sec. 2.4)
  int pp;                // 0: off
  int pp_cap;            // p-p particles a warp holds
  double beam;           // sqrt(4 pi / N_ray): beam width per unit distance
  const float* mass;     // [N] sorted
  float4* pp_xh;         // [warps][pp_cap] position, h
  float4* pp_kc;         // [warps][pp_cap] kappa_b m 3 / (pi h^2) per band
  int* pp_si;            // [warps][pp_cap] sorted element index
  float4* pp_w;          // [warps][pp_cap] per receiver: x_k - x, |x_k - x|^2 - h_k^2
  float4* pp_u;          // [warps][pp_cap] per receiver: unit x_k - x, cap threshold
  uint32_t* pp_mask;     // [warps][kCubeCells][pp_cap / 32] per receiver: the p-p
                         // particles that can meet a segment whose direction lies
                         // in each direction cell
  // directed rays (Sec. 3.4.1): the beam holding the target points at it
  int directed;
  double target[3];      // normalised
};

// The leaf holding each slot's element: down the tree by the first element
// of each upper half.
__global__ void k_bucket_leaf(const int* __restrict__ child, const int* __restrict__ first,
                              const uint64_t* __restrict__ keys, int64_t A, int64_t N,
                              int* __restrict__ leaf) {
  const int64_t p = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (p >= A) return;
  const int64_t si = int64_t(keys[p]);
  if (si >= N) {
    leaf[p] = -1;
    return;
  }
  int q = 0;
  for (int c = child[0]; c >= 0; c = child[q]) q = si < first[c + 1] ? c : c + 1;
  leaf[p] = q;
}

// The bucket's p-p radius and particles (Sec. 2.4): from the radius of the
// sphere through the leaf's corners, the radius grows to h_j / beam for the
// largest gas element j inside until nothing inside is wider than the beam
// there.  Membership is decided in FP64 on the FP64 positions.  The warp
// walks the cells that reach the sphere; lane 0 of the warp's origin slot
// gets the FP64 radius, and the particles go to the warp's p-p arrays.
// Returns their count (warp-uniform).
template <int NBP>
__device__ int collect_pp(const WalkArgs& a, const BucketArgs& bk, const double* o64, double r0,
                          int lane, int* stk, int64_t gw, double& rpp) {
  float4* xh = bk.pp_xh + gw * bk.pp_cap;
  float4* kc = bk.pp_kc + gw * bk.pp_cap;
  int* psi = bk.pp_si + gw * bk.pp_cap;
  const float3 o = make_float3(float(o64[0]), float(o64[1]), float(o64[2]));
  const unsigned lt = (1u << lane) - 1u;
  double r = r0;
  int n = 0;
  for (int it = 0; it < 64; ++it) {
    // the gas elements within r of the centre, and the largest h among them
    const float rf = float(r) * (1.0f + 1e-5f) + 1e-7f;  // box test: never too tight
    n = 0;
    float H = 0.0f;
    int sp = 1;
    if (lane == 0) stk[0] = 0;
    __syncwarp();
    while (sp > 0) {
      const int k = min(32, sp);
      const int q = lane < k ? stk[sp - 1 - lane] : -1;
      sp -= k;
      __syncwarp();
      int npush = 0, child = -1, first = 0, count = 0;
      if (q >= 0) {
        const NodeW nd = a.nodes[q];
        const float3 e = node_ext(nd.meta);
        const float dx = fmaxf(0.0f, fmaxf(nd.lo[0] - o.x, o.x - (nd.lo[0] + e.x)));
        const float dy = fmaxf(0.0f, fmaxf(nd.lo[1] - o.y, o.y - (nd.lo[1] + e.y)));
        const float dz = fmaxf(0.0f, fmaxf(nd.lo[2] - o.z, o.z - (nd.lo[2] + e.z)));
        if (dx * dx + dy * dy + dz * dz < rf * rf && nd.count > 0) {
          if (nd.meta & kMetaLeaf) {
            first = nd.aux;
            count = nd.count;
          } else {
            npush = 2;
            child = nd.child;
          }
        }
      }
      const int incl = warp_incl_scan(npush, lane);
      const int tot = __shfl_sync(0xffffffffu, incl, 31);
      if (npush) {
        const int pos = sp + incl - npush;
        if (pos + 2 <= a.stack_ints) {
          stk[pos] = child + 1;
          stk[pos + 1] = child;
        } else {
          atomicOr(a.status, kStatusStackOverflow);
        }
      }
      sp = min(sp + tot, a.stack_ints);
      int maxc = count;
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) maxc = max(maxc, __shfl_xor_sync(0xffffffffu, maxc, off));
      for (int e = 0; e < maxc; ++e) {
        bool in = false;
        const int sj = first + e;
        if (e < count && bk.mass[sj] > 0.0f) {
          const double* p = a.pos64 + 3 * int64_t(sj);
          double d2 = 0.0;
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            const double dd = __dsub_rn(p[c], o64[c]);
            d2 = __dadd_rn(d2, __dmul_rn(dd, dd));
          }
          in = sqrt(d2) < r;
        }
        const unsigned m = __ballot_sync(0xffffffffu, in);
        if (in) {
          const int idx = n + __popc(m & lt);
          const float h = a.hn[sj];
          H = fmaxf(H, h);
          if (idx < bk.pp_cap) {
            const float4 pj = a.pos32[sj];
            xh[idx] = make_float4(pj.x, pj.y, pj.z, h);
            // kappa m is in caller units, h normalised: 3/(pi h^2) in caller units
            const float c = float(3.0 / (3.14159265358979 * double(h) * double(h)) * a.inv_size2);
            float kv[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
            for (int b = 0; b < NBP; ++b) kv[b] = a.km[int64_t(sj) * NBP + b] * c;
            kc[idx] = make_float4(kv[0], kv[1], kv[2], kv[3]);
            psi[idx] = sj;
          }
        }
        n += __popc(m);
      }
      __syncwarp();
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) H = fmaxf(H, __shfl_xor_sync(0xffffffffu, H, off));
    const double grown = fmax(r, double(H) / bk.beam);
    if (grown == r) break;
    r = grown;
  }
  if (n > bk.pp_cap) {
    if (lane == 0) atomicOr(a.status, kStatusPPOverflow);
    n = bk.pp_cap;
  }
  rpp = r;
  __syncwarp();
  return n;
}

// Direction cells that cull the p-p particles per source: the six faces of
// the cube, each cut into 4 x 4 squares, projected onto the sphere.  Every
// cell lies within 0.3398 rad of its centre direction; the cap tests use
// 0.345 rad, a bound with a margin far above FP32 rounding.
constexpr int kCubeCells = 96;
constexpr float kCubeCosR = 0.941075452606513f;    // cos(0.345)
constexpr float kCubeSinR = 0.33819667724779123f;  // sin(0.345)

// The cell holding direction v (any length > 0).
__device__ __forceinline__ int cube_cell(float vx, float vy, float vz) {
  const float ax = fabsf(vx), ay = fabsf(vy), az = fabsf(vz);
  int m;
  float vm, ca, cb;
  if (ax >= ay && ax >= az) {
    m = 0; vm = vx; ca = vy; cb = vz;
  } else if (ay >= az) {
    m = 1; vm = vy; ca = vx; cb = vz;
  } else {
    m = 2; vm = vz; ca = vx; cb = vy;
  }
  const float inv = 1.0f / fabsf(vm);
  const int i = min(3, max(0, int((ca * inv + 1.0f) * 2.0f)));
  const int j = min(3, max(0, int((cb * inv + 1.0f) * 2.0f)));
  // cells of a face in Morton order of (i, j): consecutive cells are neighbours
  return (2 * m + (vm < 0.0f ? 1 : 0)) * 16 +
         ((i & 1) | ((j & 1) << 1) | ((i & 2) << 1) | ((j & 2) << 2));
}

// The unit centre direction of cell c.
__device__ __forceinline__ float3 cube_centre(int c) {
  const int f = c >> 4, m = f >> 1;
  const float sgn = (f & 1) ? -1.0f : 1.0f;
  const int mo = c & 15;
  const int ci = (mo & 1) | ((mo >> 1) & 2), cj = ((mo >> 1) & 1) | ((mo >> 2) & 2);
  const float ca = -0.75f + 0.5f * float(ci), cb = -0.75f + 0.5f * float(cj);
  const float n = rsqrtf(1.0f + ca * ca + cb * cb);
  if (m == 0) return make_float3(sgn * n, ca * n, cb * n);
  if (m == 1) return make_float3(ca * n, sgn * n, cb * n);
  return make_float3(ca * n, cb * n, sgn * n);
}

// Seen from the receiver, p-p particle k can only come within h_k of a
// segment whose direction v makes an angle below beta_k = asin(h_k / |w_k|)
// with w_k = x_k - x (or, with the receiver inside its disc, in any
// direction; the clamped ends of the segment stay inside the same cap).
// Per receiver, mask[c][g] bit i marks the particles 32 g + i whose cap,
// widened by the cell bound, reaches cell c; pu[k] holds w_k / |w_k| and
// cos(beta_k + bound).  Each lane owns cells lane, lane + 32, lane + 64.
__device__ __forceinline__ void pp_cull_masks(int npp, int lane, const float4* pw,
                                              const float4* xh, float4* pu, uint32_t* mask) {
  const int W = (npp + 31) >> 5;
  for (int k = lane; k < npp; k += 32) {
    const float4 w = pw[k];
    const float hk = xh[k].w;
    const float D2 = w.x * w.x + w.y * w.y + w.z * w.z;
    float4 u = make_float4(0.0f, 0.0f, 0.0f, -2.0f);  // every direction
    if (D2 > hk * hk * (1.0f + 1e-4f)) {
      const float iD = rsqrtf(D2);
      const float sb = fminf(1.0f, hk * iD), cb = sqrtf(fmaxf(0.0f, 1.0f - sb * sb));
      u = make_float4(w.x * iD, w.y * iD, w.z * iD, cb * kCubeCosR - sb * kCubeSinR);
    }
    pu[k] = u;
  }
  __syncwarp();
  const float3 c0 = cube_centre(lane), c1 = cube_centre(lane + 32), c2 = cube_centre(lane + 64);
  for (int g = 0; g < W; ++g) {
    uint32_t m0 = 0, m1 = 0, m2 = 0;
    const int kn = min(32, npp - 32 * g);
    for (int i = 0; i < kn; ++i) {
      const float4 u = pu[32 * g + i];
      m0 |= uint32_t(u.x * c0.x + u.y * c0.y + u.z * c0.z >= u.w) << i;
      m1 |= uint32_t(u.x * c1.x + u.y * c1.y + u.z * c1.z >= u.w) << i;
      m2 |= uint32_t(u.x * c2.x + u.y * c2.y + u.z * c2.z >= u.w) << i;
    }
    mask[lane * W + g] = m0;
    mask[(lane + 32) * W + g] = m1;
    mask[(lane + 64) * W + g] = m2;
  }
  __syncwarp();
}

// What pp_term reads of p-p particle k: its offset from the receiver, its
// position and h, its column factors per band, its sorted index.
struct PPData {
  float4 w, q, c;
  int kk;
};

__device__ __forceinline__ PPData pp_load(int k, const float4* pw, const float4* xh,
                                          const float4* kc, const int* psi) {
  PPData d;
  d.w = pw[k];
  d.kk = psi[k];
  d.q = xh[k];
  d.c = kc[k];
  return d;
}

// One p-p particle k's optical depth, per band, added to tau for the
// segment from a receiver at x (sorted index si) to a source at p (its
// element sj, or -1), v = p - x, r2 = |v|^2: the particle counts when it is
// neither of the two, lies closer to the source than the receiver and
// within h_k of the segment (distance b), and adds kappa_k 3 m_k /
// (pi h_k^2) (1 - b / h_k).  pw[k] = (w, |w|^2 - h_k^2) with w = x_k - x,
// set per receiver: with t the clamped segment parameter of the closest
// point, |w|^2 - b^2 = t (2 w.v - t r^2).  The column goes to zero at
// b = h_k, so that test needs no care; "closer" is decided in FP32 and
// again in FP64 (positions pos64 of the receiver, p64 of the source) inside
// a guard band that covers the FP32 error.  Lanes that are not live (no
// source) add zero.  Every lane of the warp calls it for the same k (a vote
// skips the rest when no lane's segment meets the particle).
template <int NBP>
__device__ __forceinline__ void pp_term(const WalkArgs& a, const PPData& d, bool live, int si,
                                        float4 p, const double* p64, int sj, float vx, float vy,
                                        float vz, float r, float r2, float ir2, float guard,
                                        float* tau) {
  const float4 w = d.w;
  const int kk = d.kk;
  const float4 q = d.q;
  const float4 c = d.c;
  const float dot = w.x * vx + w.y * vy + w.z * vz;
  const float t = fminf(fmaxf(dot * ir2, 0.0f), 1.0f);
  const float g = t * (2.0f * dot - t * r2);  // |w|^2 - b^2
  bool hit = live && (g > w.w) && kk != si && kk != sj;  // b < h_k, not the pair itself
  if (!__any_sync(0xffffffffu, hit)) return;  // no lane's segment meets the particle
  const float dx = q.x - p.x, dy = q.y - p.y, dz = q.z - p.z;
  const float dj2 = dx * dx + dy * dy + dz * dz;
  const bool clear = fabsf(r2 - dj2) > guard * (r + sqrtf(dj2));
  bool front = dj2 < r2;
  if (hit && !clear) {  // FP64: |x_k - p| < |x - p|
    const double* xk = a.pos64 + 3 * int64_t(kk);
    const double* xi = a.pos64 + 3 * int64_t(si);
    double d2k = 0.0, d2i = 0.0;
    for (int cc = 0; cc < 3; ++cc) {
      const double dk = __dsub_rn(xk[cc], p64[cc]);
      const double di = __dsub_rn(xi[cc], p64[cc]);
      d2k = __dadd_rn(d2k, __dmul_rn(dk, dk));
      d2i = __dadd_rn(d2i, __dmul_rn(di, di));
    }
    front = sqrt(d2k) < sqrt(d2i);
  }
  hit = hit && front;
  const float b2 = fmaxf(0.0f, (w.w + q.w * q.w) - g);
  const float f = hit ? fmaxf(0.0f, 1.0f - sqrtf(b2) / q.w) : 0.0f;
  const float cv[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
  for (int bb = 0; bb < NBP; ++bb) tau[bb] += cv[bb] * f;
}

// The n staged sources of a bucket in the order of their direction cell
// seen from the bucket centre o, into perm (a stable counting sort: cell,
// then index), so that the 32 sources a warp evaluates together point in
// few directions.  cnt is shared memory of at least kCubeCells ints; with
// fewer (nside 1) the order is left as it is.
__device__ __forceinline__ void sort_sources_by_cell(const WalkArgs& a, int lane,
                                                     const SrcEntry* V, int n, float3 o,
                                                     int* cnt, int cnt_ints, int* perm) {
  if (cnt_ints < kCubeCells) {
    for (int e = lane; e < n; e += 32) perm[e] = e;
    __syncwarp();
    return;
  }
  auto cell_of = [&](int e) {
    const int ref = V[e].ref;
    const float4 pj = (ref & kRefElement) ? a.pos32[ref & 0x7fffffff] : a.csrc[ref];
    return cube_cell(pj.x - o.x, pj.y - o.y, pj.z - o.z);
  };
  for (int c = lane; c < kCubeCells; c += 32) cnt[c] = 0;
  __syncwarp();
  for (int e = lane; e < n; e += 32) atomicAdd(&cnt[cell_of(e)], 1);
  __syncwarp();
  const int c0 = 3 * lane;  // 96 = 3 x 32 cells
  const int s0 = cnt[c0], s1 = cnt[c0 + 1], s2 = cnt[c0 + 2];
  const int incl = warp_incl_scan(s0 + s1 + s2, lane);
  const int base = incl - (s0 + s1 + s2);
  __syncwarp();
  cnt[c0] = base;
  cnt[c0 + 1] = base + s0;
  cnt[c0 + 2] = base + s0 + s1;
  __syncwarp();
  const unsigned lt = (1u << lane) - 1u;
  for (int e0 = 0; e0 < n; e0 += 32) {
    const int e = e0 + lane;
    const bool in = e < n;
    const int c = in ? cell_of(e) : kCubeCells + lane;  // idle lanes match nothing
    const unsigned peers = __match_any_sync(0xffffffffu, c);
    const int rank = __popc(peers & lt);
    const int slot = in ? cnt[c] + rank : 0;
    __syncwarp();
    if (in && rank == 0) cnt[c] += __popc(peers);
    __syncwarp();
    if (in) perm[slot] = e;
  }
  __syncwarp();
}

// The staged sources against the bucket's receivers (one per lane j < nrec,
// position xr, size hr, sorted index sir): per receiver, all lanes over the
// sources with a compensated FP32 sum, reduced in FP64 into acc of lane j.
// (Without p-p absorption; eval_bucket_pp adds it.)
template <int NBP>
__device__ __forceinline__ void eval_bucket(const WalkArgs& a, bool soft, int lane,
                                            const SrcEntry* V, const float* T, int n, int nrec,
                                            float4 xr, float hr, int sir, double* acc) {
  for (int j = 0; j < nrec; ++j) {
    const float xx = __shfl_sync(0xffffffffu, xr.x, j);
    const float xy = __shfl_sync(0xffffffffu, xr.y, j);
    const float xz = __shfl_sync(0xffffffffu, xr.z, j);
    const float hh = __shfl_sync(0xffffffffu, hr, j);
    const int si = __shfl_sync(0xffffffffu, sir, j);
    float Js[NBP], Jc[NBP];
#pragma unroll
    for (int b = 0; b < NBP; ++b) Js[b] = Jc[b] = 0.0f;
    for (int e = lane; e < n; e += 32) {
      const SrcEntry src = V[e];
      const bool elem = (src.ref & kRefElement) != 0;
      const int64_t id = src.ref & 0x7fffffff;
      const float4 p = elem ? a.pos32[id] : a.csrc[id];
      const float vx = p.x - xx, vy = p.y - xy, vz = p.z - xz;
      const float r2 = vx * vx + vy * vy + vz * vz;
      if (!(r2 > 0.0f)) continue;  // the receiver itself, or on top of it
      const float r = sqrtf(r2);
      const float w = soft ? soft_kernel(r, hh) : 1.0f / (kFourPi * r2);
      const float rs = r / src.w;  // w: the source's projected distance
      const BandVec<NBP> L = load_bands<NBP>(elem ? a.Lelem + id * NBP : a.Lnode + id * NBP);
      const BandVec<NBP> tk = load_bands<NBP>(T + int64_t(e) * NBP);
#pragma unroll
      for (int b = 0; b < NBP; ++b) {
        const float term = L.v[b] * w * expf(-(tk.v[b] * rs));
        const float y = term - Jc[b];
        const float t = Js[b] + y;
        Jc[b] = (t - Js[b]) - y;
        Js[b] = t;
      }
    }
#pragma unroll
    for (int b = 0; b < NBP; ++b) {
      double v = double(Js[b]) - double(Jc[b]);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == j) acc[b] += v;
    }
  }
}

// eval_bucket with the p-p absorption of Sec. 2.4.  Per receiver the p-p
// particles' offsets and direction masks are set up (pp_cull_masks); the
// sources, in the order perm (grouped by direction cell), are evaluated 32
// at a time.  A group walks, in increasing k, the particles that the
// direction cell of any of its sources can reach: for each source these
// include every particle that can absorb on its segment, and the others
// add nothing, so each source's p-p optical depth is the sum over all
// particles in index order.
template <int NBP>
__device__ __forceinline__ void eval_bucket_pp(const WalkArgs& a, bool soft, int lane,
                                               const SrcEntry* V, const float* T, const int* perm,
                                               int n, int nrec, float4 xr, float hr, int sir,
                                               double* acc, int npp, const float4* ppxh,
                                               const float4* ppkc, const int* ppsi, float4* ppw,
                                               float4* ppu, uint32_t* ppmask) {
  const int W = (npp + 31) >> 5;
  for (int j = 0; j < nrec; ++j) {
    const float xx = __shfl_sync(0xffffffffu, xr.x, j);
    const float xy = __shfl_sync(0xffffffffu, xr.y, j);
    const float xz = __shfl_sync(0xffffffffu, xr.z, j);
    const float hh = __shfl_sync(0xffffffffu, hr, j);
    const int si = __shfl_sync(0xffffffffu, sir, j);
    for (int k = lane; k < npp; k += 32) {  // the p-p particles seen from this receiver
      const float4 q = ppxh[k];
      const float wx = q.x - xx, wy = q.y - xy, wz = q.z - xz;
      ppw[k] = make_float4(wx, wy, wz, (wx * wx + wy * wy + wz * wz) - q.w * q.w);
    }
    __syncwarp();
    pp_cull_masks(npp, lane, ppw, ppxh, ppu, ppmask);
    float Js[NBP], Jc[NBP];
#pragma unroll
    for (int b = 0; b < NBP; ++b) Js[b] = Jc[b] = 0.0f;
    for (int e0 = 0; e0 < n; e0 += 32) {
      const int e = e0 + lane < n ? perm[e0 + lane] : -1;
      bool live = false, elem = false;
      int64_t id = 0;
      float4 p = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
      float vx = 0.0f, vy = 0.0f, vz = 0.0f, r = 1.0f, w = 0.0f, s_proj = 1.0f;
      if (e >= 0) {
        const SrcEntry src = V[e];
        elem = (src.ref & kRefElement) != 0;
        id = src.ref & 0x7fffffff;
        p = elem ? a.pos32[id] : a.csrc[id];
        vx = p.x - xx;
        vy = p.y - xy;
        vz = p.z - xz;
        const float rr = vx * vx + vy * vy + vz * vz;
        live = rr > 0.0f;  // else the receiver itself, or on top of it
        if (live) {
          r = sqrtf(rr);
          w = soft ? soft_kernel(r, hh) : 1.0f / (kFourPi * rr);
          s_proj = src.w;  // the source's projected distance
        }
      }
      const float r2 = r * r, ir2 = 1.0f / r2, guard = 2e-6f * r + 1e-7f;
      const double* p64 = elem ? a.pos64 + 3 * id : a.c64 + 3 * id;
      const int sj = elem ? int(id) : -1;
      const int cell = live ? cube_cell(vx, vy, vz) : 0;
      float tpp[NBP];
#pragma unroll
      for (int b = 0; b < NBP; ++b) tpp[b] = 0.0f;
      for (int g = 0; g < W; ++g) {
        uint32_t bits = live ? ppmask[cell * W + g] : 0u;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) bits |= __shfl_xor_sync(0xffffffffu, bits, o);
        while (bits) {  // two particles at a time: both loads in flight together
          const int k0 = 32 * g + __ffs(bits) - 1;
          bits &= bits - 1u;
          const bool two = bits != 0u;
          const int k1 = two ? 32 * g + __ffs(bits) - 1 : k0;
          if (two) bits &= bits - 1u;
          const PPData d0 = pp_load(k0, ppw, ppxh, ppkc, ppsi);
          const PPData d1 = pp_load(k1, ppw, ppxh, ppkc, ppsi);
          pp_term<NBP>(a, d0, live, si, p, p64, sj, vx, vy, vz, r, r2, ir2, guard, tpp);
          if (two) pp_term<NBP>(a, d1, live, si, p, p64, sj, vx, vy, vz, r, r2, ir2, guard, tpp);
        }
      }
      if (live) {
        const float rs = r / s_proj;
        const BandVec<NBP> L = load_bands<NBP>(elem ? a.Lelem + id * NBP : a.Lnode + id * NBP);
        const BandVec<NBP> tk = load_bands<NBP>(T + int64_t(e) * NBP);
#pragma unroll
        for (int b = 0; b < NBP; ++b) {
          const float term = L.v[b] * w * expf(-(tk.v[b] * rs + tpp[b]));
          const float y = term - Jc[b];
          const float t = Js[b] + y;
          Jc[b] = (t - Js[b]) - y;
          Js[b] = t;
        }
      }
    }
#pragma unroll
    for (int b = 0; b < NBP; ++b) {
      double v = double(Js[b]) - double(Jc[b]);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == j) acc[b] += v;
    }
    __syncwarp();  // ppw, ppu, ppmask are rewritten for the next receiver
  }
}

// J of the receivers in slots [p0, p1), all in leaf q, into their rows
// (kPP: with the p-p absorption of Sec. 2.4; kCSM: with the complex source
// model of Sec. 2.7).
template <int NBP, bool kPP, bool kCSM>
__device__ void walk_bucket(const WalkArgs& a, const BucketArgs& bk, int64_t p0, int64_t p1,
                            int q, int64_t gw, int lane, int* stk, int* off, int* next_beam,
                            int* lstk, SrcEntry* U, int* Up, SrcEntry* V, float* T) {
  if (q < 0) {  // receivers outside [0, N): NaN rows and a status bit
    for (int64_t p = p0 + lane; p < p1; p += 32)
      for (int c = 0; c < a.nbsel; ++c) a.J[int64_t(a.order[p]) * a.nbsel + c] = __int_as_float(0x7fc00000);
    if (lane == 0) atomicOr(a.status, kStatusBadActive);
    return;
  }
  const NodeW lf = a.nodes[q];
  const float3 e = node_ext(lf.meta);
  // the box centre: lo + ext/2 is a multiple of 2^-22 in [0, 1), exact in FP32
  const float3 o = make_float3(lf.lo[0] + 0.5f * e.x, lf.lo[1] + 0.5f * e.y, lf.lo[2] + 0.5f * e.z);
  const int si_o = int(-1 - gw);  // the warp's origin slot (origin64<true>)
  if (lane == 0) {
    double* o64 = a.origin64 + kOriginWords * gw;
    o64[0] = double(o.x);
    o64[1] = double(o.y);
    o64[2] = double(o.z);
    o64[3] = 0.0;
    o64[7] = -1.0;
    if (bk.directed) {  // Sec. 3.4.1: the beam holding the target points at it
      const double vx = bk.target[0] - o64[0], vy = bk.target[1] - o64[1],
                   vz = bk.target[2] - o64[2];
      const double nv = sqrt(vx * vx + vy * vy + vz * vz);
      if (nv > 0.0) {
        o64[4] = vx / nv;
        o64[5] = vy / nv;
        o64[6] = vz / nv;
        o64[7] = double(hp_vec2pix_f64(a.nside, vx, vy, vz));
      }
    }
  }
  NodeW* chain = reinterpret_cast<NodeW*>(off + 2 * a.npix + 36);
  const int leaf = build_chain(a.nodes, o, lane, chain);  // == q
  const bool soft = (bk.rflags & TREVR2_SOFT) != 0;
  // Sec. 2.4: the bucket's p-p radius and particles
  int npp = 0;
  float rpp = 0.0f;
  if constexpr (kPP) {
    const double r0 = 0.5 * sqrt(double(e.x) * e.x + double(e.y) * e.y + double(e.z) * e.z);
    double r64 = 0.0;
    __syncwarp();
    npp = collect_pp<NBP>(a, bk, a.origin64 + kOriginWords * gw, r0, lane, stk, gw, r64);
    if (lane == 0) a.origin64[kOriginWords * gw + 3] = r64;
    rpp = float(r64);
    __syncwarp();
  }
  const float4* ppxh = bk.pp_xh + gw * bk.pp_cap;
  const float4* ppkc = bk.pp_kc + gw * bk.pp_cap;
  const int* ppsi = bk.pp_si + gw * bk.pp_cap;
  float4* ppw = bk.pp_w + gw * bk.pp_cap;
  float4* ppu = bk.pp_u + gw * bk.pp_cap;
  uint32_t* ppmask = bk.pp_mask + gw * int64_t(kCubeCells) * (bk.pp_cap / 32);
  for (int64_t c0 = p0; c0 < p1; c0 += 32) {
    const int nrec = int(min(int64_t(32), p1 - c0));
    int si = -1;
    float4 xr = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    float hr = 1.0f;
    if (lane < nrec) {
      si = int(bk.keys[c0 + lane]);
      xr = a.pos32[si];
      hr = a.hn[si];
    }
    double acc[NBP];
#pragma unroll
    for (int b = 0; b < NBP; ++b) acc[b] = 0.0;
    for (int lo = 0;; lo += a.M) {
      const int total = phase_sources<true, kPP>(a, o, si_o, lane, stk, a.src_stack_cap, U, Up, lo,
                                                 rpp);
      const int staged = min(total - lo, a.M);
      make_sources<true, kCSM>(a, o, si_o, lane, U, Up, staged);
      const int n = staged > 0 ? bin_sources(a, lane, U, Up, staged, V, off) : 0;
      if (n > 0) {
        int* order = off + a.npix;
        const int nbeams = order_beams(a, lane, V, off, order, order + a.npix);
        if (lane == 0) *next_beam = 32;
        __syncwarp();
        phase_absorb<NBP, true, kPP, kCSM>(a, o, si_o, lane, lstk, V, T, off, order, nbeams,
                                           next_beam, chain, leaf, rpp);
        __syncwarp();
        if constexpr (kPP) {
          // Up, the staged records' beams, is free once they are binned
          sort_sources_by_cell(a, lane, V, n, o, off, 2 * a.npix + 32, Up);
          eval_bucket_pp<NBP>(a, soft, lane, V, T, Up, n, nrec, xr, hr, si, acc, npp, ppxh, ppkc,
                              ppsi, ppw, ppu, ppmask);
        } else {
          eval_bucket<NBP>(a, soft, lane, V, T, n, nrec, xr, hr, si, acc);
        }
        __syncwarp();
      }
      if (lo + a.M >= total) break;
    }
    if (lane < nrec) {
      float* Jrow = a.J + int64_t(a.order[c0 + lane]) * a.nbsel;
      for (int c = 0; c < a.nbsel; ++c) {
        const int b = a.bsel[c];
        double v = 0.0;
#pragma unroll
        for (int d = 0; d < NBP; ++d)
          if (d == b) v = acc[d];
        v *= a.inv_size2;
        if (bk.rflags & TREVR2_THICK) {
          const double h = double(hr) * a.size;
          const double tau = double(a.km[int64_t(si) * NBP + b]) / (h * h);
          if (tau > 0.0) v *= -expm1(-tau) / tau;
        }
        Jrow[c] = float(v);
      }
    }
  }
}

// One warp per bucket; slots from a global counter.
// Blocks per SM the per-bucket walk with p-p absorption is compiled for:
// its particle loop holds two particles' loads in flight, and 5 blocks (96
// registers a thread) measured faster than 7 (72, spilling) and than 4 or 6.
constexpr int kPPBlocksPerSM = 5;

template <int NBP, int WARPS, bool kPP, bool kCSM>
__global__ void __launch_bounds__(WARPS * 32, kPP ? kPPBlocksPerSM : kWalkWarpsPerSM / WARPS)
    k_walk_bucket(WalkArgs a, const __grid_constant__ BucketArgs bk) {
  init_ext_tab();
  extern __shared__ int smem[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t gw = int64_t(blockIdx.x) * WARPS + wib;
  int* wsm = smem + wib * (a.stack_ints + 2 * a.npix + 36 + 8 * (a.max_depth + 1));
  int* stk = wsm;
  int* off = wsm + a.stack_ints;
  int* next_beam = off + 2 * a.npix + 32;
  int* lstk = stk + lane * 2 * (a.max_depth + 2);
  SrcEntry* U = a.srcU + gw * a.M;
  int* Up = a.pixU + gw * a.M;
  SrcEntry* V = a.srcV + gw * a.M;
  float* T = a.srcT + gw * a.M * 4;
  for (;;) {
    unsigned long long slot = 0;
    if (lane == 0) slot = atomicAdd(a.counter, 1ull);
    slot = __shfl_sync(0xffffffffu, slot, 0);
    if (slot >= (unsigned long long)a.A) break;
    const int64_t p0 = int64_t(slot);
    const int q = bk.leaf[p0];
    if (p0 > 0 && bk.leaf[p0 - 1] == q) continue;  // not the first slot of its bucket
    // the bucket's end: the first later slot in another leaf
    int64_t p1 = p0 + 1;
    for (;;) {
      const int64_t p = p1 + lane;
      const unsigned same = __ballot_sync(0xffffffffu, p < a.A && bk.leaf[p] == q);
      if (same == 0xffffffffu) {
        p1 += 32;
        continue;
      }
      p1 += __ffs(~same) - 1;
      break;
    }
    walk_bucket<NBP, kPP, kCSM>(a, bk, p0, p1, q, gw, lane, stk, off, next_beam, lstk, U, Up, V,
                                T);
  }
}

// Many receiver subsets over several trees in one launch (individual
// timesteps over independent snapshots, Sec. 1.2 and Sec. 3.1): row r of the
// concatenated list belongs to the subset s with offsets[s] <= r <
// offsets[s + 1] and is walked in tree tree_of[s].  Rows that ask for the
// same receiver of the same tree get the same J, so a run walks every
// distinct (tree, receiver) once, in the tree's Morton order, and copies the
// row: keys (tree, element position in the tree), sorted with their rows,
// first of each key marked and numbered by a scan, the distinct keys walked,
// the results scattered back.
constexpr int kMaxBatchTrees = TREVR2_MAX_BATCH_TREES;

struct BatchArgs {
  WalkArgs tree[kMaxBatchTrees];  // per-tree arguments (their active/J fields unused)
  int ntrees;
  int key_shift;                  // key = tree << key_shift | element position
  const int64_t* active;          // [total] concatenated receiver indices
  const int64_t* offsets;         // [nsub + 1]
  const int* tree_of;             // [nsub]
  int nsub;
  int64_t total;                  // rows of this run
  float* J;                       // [total][nbsel]
  int nbsel;
  uint64_t* keys;                 // [total] keys of the rows, sorted
  int* rows;                      // [total] row of each sorted key
  int* first_scan;                // [total] distinct keys before each sorted key
  uint64_t* ukeys;                // [distinct] the distinct keys
  float* Ju;                      // [distinct][nbsel] J of each distinct key
  int* n_distinct;                // device count of distinct keys
  SrcEntry* srcU;
  int* pixU;
  SrcEntry* srcV;
  float* srcT;
  int M;
  int stack_ints;
  int npix;
  int max_depth;
  unsigned long long* counter;
  // per-bucket plans (TREVR2_BUCKET): for each distinct key, its sorted
  // element index, its (tree, leaf) and its own row of Ju
  uint64_t* usi;                  // [total]
  uint64_t* ubkey;                // [total] tree << 32 | leaf (invalid: ntrees << 32)
  int* uorder;                    // [total] identity
  int* tree_range;                // [ntrees + 1] first distinct key of each tree
};

// What one tree's launch of a batch run needs besides the tree's own walk
// arguments: its range of the distinct keys, where their rows go, the walk
// buffers and the work counter.
struct BatchSlice {
  const uint64_t* ukeys;
  const uint64_t* ubkey;
  const int* tree_range;
  float* Ju;
  int t;
  int key_shift;
  int nbsel;
  SrcEntry* srcU;
  int* pixU;
  SrcEntry* srcV;
  float* srcT;
  unsigned long long* counter;
};

// Per-tree arguments of a per-bucket plan: the bucket walk's own arguments
// and the topology that finds each receiver's leaf.
struct BucketBatchArgs {
  BucketArgs tree[kMaxBatchTrees];
  const int* child[kMaxBatchTrees];
  const int* first[kMaxBatchTrees];
};

// Key of every row: its tree and the receiver's position in that tree's
// element order; invalid receivers get tree = ntrees (sorted last, one key
// per row) and their tree's status bit.
__global__ void k_batch_keys(const __grid_constant__ BatchArgs B) {
  const int64_t r = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (r >= B.total) return;
  int lo = 0, hi = B.nsub;  // offsets[lo] <= r < offsets[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (B.offsets[mid] <= r) lo = mid; else hi = mid;
  }
  const int t = B.tree_of[lo];
  const WalkArgs& a = B.tree[t];
  const int64_t io = B.active[r];
  if (io >= 0 && io < a.N) {
    B.keys[r] = (uint64_t(t) << B.key_shift) | uint64_t(uint32_t(a.inv[io]));
  } else {
    B.keys[r] = uint64_t(B.ntrees) << B.key_shift;
    atomicOr(a.status, kStatusBadActive);
  }
  B.rows[r] = int(r);
}

__device__ __forceinline__ bool first_of_key(const uint64_t* keys, int64_t p) {
  return p == 0 || keys[p] != keys[p - 1];
}

__global__ void k_batch_first(const __grid_constant__ BatchArgs B) {
  const int64_t p = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (p < B.total) B.first_scan[p] = first_of_key(B.keys, p) ? 1 : 0;
}

__global__ void k_batch_distinct(const __grid_constant__ BatchArgs B) {
  const int64_t p = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (p < B.total && first_of_key(B.keys, p)) B.ukeys[B.first_scan[p]] = B.keys[p];
}

// Every row gets its key's J (NaN for an invalid receiver).
__global__ void k_batch_scatter(const __grid_constant__ BatchArgs B) {
  const int64_t p = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (p >= B.total) return;
  const uint64_t key = B.keys[p];
  const int64_t r = B.rows[p];
  const int64_t u = B.first_scan[p] - (first_of_key(B.keys, p) ? 0 : 1);
  const bool ok = int(key >> B.key_shift) < B.ntrees;
  for (int j = 0; j < B.nbsel; ++j)
    B.J[r * B.nbsel + j] = ok ? B.Ju[u * B.nbsel + j] : __int_as_float(0x7fc00000);
}

// The range of each tree among the distinct keys (sorted by tree, invalid
// receivers last): tree_range[t] is the first key of tree t or later.
__global__ void k_batch_tree_range(const __grid_constant__ BatchArgs B) {
  const int t = threadIdx.x;
  if (t > B.ntrees) return;
  int lo = 0, hi = *B.n_distinct;
  const uint64_t key = uint64_t(t) << B.key_shift;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (B.ukeys[mid] < key) lo = mid + 1; else hi = mid;
  }
  B.tree_range[t] = lo;
}

// One launch per tree (its walk arguments are this launch's own parameter,
// so the walk reads them as directly as k_walk does): one warp per distinct
// key of the tree, keys from a global counter.
template <int NBP, int WARPS>
__global__ void __launch_bounds__(WARPS * 32, kWalkWarpsPerSM / WARPS)
    k_walk_batched(WalkArgs a, const __grid_constant__ BatchSlice S) {
  init_ext_tab();
  extern __shared__ int smem[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t gw = int64_t(blockIdx.x) * WARPS + wib;
  int* wsm = smem + wib * (a.stack_ints + 2 * a.npix + 36 + 8 * (a.max_depth + 1));
  int* stk = wsm;
  int* off = wsm + a.stack_ints;
  int* next_beam = off + 2 * a.npix + 32;  // after the beam order and its counts
  int* lstk = stk + lane * 2 * (a.max_depth + 2);
  SrcEntry* U = S.srcU + gw * a.M;
  int* Up = S.pixU + gw * a.M;
  SrcEntry* V = S.srcV + gw * a.M;
  float* T = S.srcT + gw * a.M * 4;
  const int64_t u0 = S.tree_range[S.t], u1 = S.tree_range[S.t + 1];
  const uint64_t mask = (uint64_t(1) << S.key_shift) - 1;
  for (;;) {
    unsigned long long slot = 0;
    if (lane == 0) slot = atomicAdd(S.counter, 1ull);
    slot = __shfl_sync(0xffffffffu, slot, 0);
    const int64_t u = u0 + int64_t(slot);
    if (u >= u1) break;
    walk_receiver_si<NBP>(a, int(S.ukeys[u] & mask), S.Ju + u * S.nbsel, lane, stk, off,
                          next_beam, lstk, U, Up, V, T);
  }
}

// Per-bucket plans: the leaf of every distinct (tree, receiver) key, down the
// tree by the first element of each upper half.  Distinct keys are sorted by
// (tree, element position), so a bucket's receivers are adjacent.
__global__ void k_batch_leaf(const __grid_constant__ BatchArgs B,
                             const __grid_constant__ BucketBatchArgs bb) {
  const int64_t u = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (u >= int64_t(*B.n_distinct)) return;
  const uint64_t key = B.ukeys[u];
  const int t = int(key >> B.key_shift);
  B.uorder[u] = int(u);
  if (t >= B.ntrees) {
    B.ubkey[u] = uint64_t(B.ntrees) << 32;
    B.usi[u] = 0;
    return;
  }
  const int si = int(key & ((uint64_t(1) << B.key_shift) - 1));
  const int* child = bb.child[t];
  const int* first = bb.first[t];
  int q = 0;
  for (int c = child[0]; c >= 0; c = child[q]) q = si < first[c + 1] ? c : c + 1;
  B.ubkey[u] = (uint64_t(t) << 32) | uint64_t(uint32_t(q));
  B.usi[u] = uint64_t(si);
}

// One warp per bucket of one tree's distinct keys (the paper's per-bucket
// walk over many subsets and snapshots), one launch per tree as for
// k_walk_batched; slots from a global counter, a bucket walked by the warp
// that takes its first slot.
template <int NBP, int WARPS, bool kPP, bool kCSM>
__global__ void __launch_bounds__(WARPS * 32, kPP ? kPPBlocksPerSM : kWalkWarpsPerSM / WARPS)
    k_walk_bucket_batched(WalkArgs a, const __grid_constant__ BucketArgs bk,
                          const __grid_constant__ BatchSlice S) {
  init_ext_tab();
  extern __shared__ int smem[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t gw = int64_t(blockIdx.x) * WARPS + wib;
  int* wsm = smem + wib * (a.stack_ints + 2 * a.npix + 36 + 8 * (a.max_depth + 1));
  int* stk = wsm;
  int* off = wsm + a.stack_ints;
  int* next_beam = off + 2 * a.npix + 32;
  int* lstk = stk + lane * 2 * (a.max_depth + 2);
  SrcEntry* U = S.srcU + gw * a.M;
  int* Up = S.pixU + gw * a.M;
  SrcEntry* V = S.srcV + gw * a.M;
  float* T = S.srcT + gw * a.M * 4;
  const int64_t u0 = S.tree_range[S.t], u1 = S.tree_range[S.t + 1];
  for (;;) {
    unsigned long long slot = 0;
    if (lane == 0) slot = atomicAdd(S.counter, 1ull);
    slot = __shfl_sync(0xffffffffu, slot, 0);
    const int64_t p0 = u0 + int64_t(slot);
    if (p0 >= u1) break;
    const uint64_t bkey = S.ubkey[p0];
    if (p0 > u0 && S.ubkey[p0 - 1] == bkey) continue;  // not the first slot of its bucket
    int64_t p1 = p0 + 1;
    for (;;) {
      const int64_t p = p1 + lane;
      const unsigned same = __ballot_sync(0xffffffffu, p < u1 && S.ubkey[p] == bkey);
      if (same == 0xffffffffu) {
        p1 += 32;
        continue;
      }
      p1 += __ffs(~same) - 1;
      break;
    }
    walk_bucket<NBP, kPP, kCSM>(a, bk, p0, p1, int(uint32_t(bkey)), gw, lane, stk, off,
                                next_beam, lstk, U, Up, V, T);
  }
}

bool valid_nside(int nside) {
  return nside >= 1 && nside <= TREVR2_MAX_NSIDE && (nside & (nside - 1)) == 0;
}

// Per-tree walk arguments for one nside (everything but the receivers, the
// output and the buffers).
void fill_walk_args(const Tree* t, const Table* tb, int nside, float theta, const int* bsel,
                    int nbsel, uint32_t flags, int M, WalkArgs* a) {
  std::memset(a, 0, sizeof(WalkArgs));
  a->nodes = t->refine_on ? t->nodes_refined : t->nodes;
  a->csrc = t->csrc;
  a->c64 = t->c64;
  a->B64 = t->B64;
  a->Lnode = t->Lnode;
  a->alpha_leaf = t->alpha_leaf;
  a->alpha_tab = tb->alpha;
  a->pos32 = t->pos32;
  a->pos64 = t->pos64;
  a->Lelem = t->Lelem;
  a->inv = t->inv;
  a->hn = t->hn;
  a->km = t->km;
  a->dirs = tb->dirs;
  a->N = t->N;
  a->nside = nside;
  a->npix = 12 * nside * nside;
  a->P = a->npix / 2;
  a->theta = theta;
  a->theta2 = theta * theta;
  a->theta64 = double(theta);
  a->guard_abs = 2e-7f * theta + 2e-7f;
  a->guard_rel = 2e-6f;
  a->flags = flags;
  a->nb = t->nb;
  a->nbsel = nbsel;
  for (int b = 0; b < TREVR2_MAX_BANDS; ++b) a->bsel[b] = b < nbsel ? bsel[b] : 0;
  a->inv_size2 = 1.0 / (t->size * t->size);
  a->size = t->size;
  a->M = M;
  a->max_depth = t->max_depth;
  a->stack_ints = 64 * (t->max_depth + 2);
  a->src_stack_cap = a->stack_ints;
  if (const int cap = debug_source_stack_cap()) a->src_stack_cap = std::min(cap, a->stack_ints);
  a->status = t->status;
  a->counter = t->counter;
}

template <int NBP>
static const void* walk_kernel_nbp(int warps, bool batched) {
  if (batched)
    return warps == 4 ? reinterpret_cast<const void*>(&k_walk_batched<NBP, 4>)
                      : reinterpret_cast<const void*>(&k_walk_batched<NBP, 8>);
  return warps == 4 ? reinterpret_cast<const void*>(&k_walk<NBP, 4>)
                    : reinterpret_cast<const void*>(&k_walk<NBP, 8>);
}

static const void* walk_kernel(int nbp, int warps, bool batched) {
  return nbp == 1 ? walk_kernel_nbp<1>(warps, batched)
       : nbp == 2 ? walk_kernel_nbp<2>(warps, batched)
                  : walk_kernel_nbp<4>(warps, batched);
}


// Shared memory attribute and resident blocks per SM of a walk kernel.
int config_walk_kernel(const void* fn, int warps, size_t smem, int* per_sm, int* sms) {
  int dev = 0, max_smem = 0;
  T2_CUDA(cudaGetDevice(&dev));
  T2_CUDA(cudaDeviceGetAttribute(sms, cudaDevAttrMultiProcessorCount, dev));
  T2_CUDA(cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  if (smem > size_t(max_smem)) {
    set_error("trevr2: the walk needs %zu bytes of shared memory per block (tree too deep for "
              "this nside)", smem);
    return TREVR2_EUNSUPPORTED;
  }
  T2_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
  *per_sm = 0;
  T2_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, fn, warps * 32, smem));
  if (*per_sm < 1) *per_sm = 1;
  return TREVR2_OK;
}

// Walk buffers: per warp, M source records in and out and their beams; the
// optical depths of the binned records reuse the space of the unbinned ones.
static size_t walk_buffer_bytes(size_t warps, int M) {
  return warps * size_t(M) * (2 * sizeof(SrcEntry) + sizeof(int));
}

static void place_walk_buffers(char* base, size_t warps, int M, SrcEntry** U, SrcEntry** V,
                               float** T, int** Up) {
  *U = reinterpret_cast<SrcEntry*>(base);
  *V = reinterpret_cast<SrcEntry*>(base + warps * M * sizeof(SrcEntry));
  *T = reinterpret_cast<float*>(*U);  // the staged records are dead once binned
  *Up = reinterpret_cast<int*>(base + 2 * warps * M * sizeof(SrcEntry));
}

// A grown-on-demand device buffer: at least `need` bytes in *buf.  A failed
// allocation leaves it empty (NULL, 0 bytes), never pointing at freed memory.
static int grow_buffer(void** buf, size_t* bytes, size_t need, cudaStream_t st, const char* what) {
  if (*bytes >= need) return TREVR2_OK;
  if (*buf) cudaFreeAsync(*buf, st);
  *buf = nullptr;
  *bytes = 0;
  T2_CHECK(device_alloc(buf, need, st, what));
  *bytes = need;
  return TREVR2_OK;
}

__global__ void k_order_keys(const int64_t* __restrict__ active, int64_t A, int64_t N,
                             const int* __restrict__ inv, uint64_t* __restrict__ keys,
                             int* __restrict__ slots) {
  const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (i >= A) return;
  const int64_t io = active[i];
  keys[i] = (io >= 0 && io < N) ? uint64_t(inv[io]) : uint64_t(N);
  slots[i] = int(i);
}

static int launch_walk(Tree* t, Table* tb, const int64_t* active, int64_t A, int nside,
                       float theta, const int* bsel, int nbsel, uint32_t flags, float* J,
                       cudaStream_t st) {
  WalkArgs a;
  fill_walk_args(t, tb, nside, theta, bsel, nbsel, flags, kSrcCapacity, &a);
  a.active = active;
  a.A = A;
  a.J = J;
  if (A > 1) {
    const size_t need = size_t(A) * (sizeof(uint64_t) + sizeof(int));
    T2_CHECK(grow_buffer(&t->order_buf, &t->order_bytes, need, st, "receiver order"));
    uint64_t* keys = static_cast<uint64_t*>(t->order_buf);
    int* slots = reinterpret_cast<int*>(keys + A);
    k_order_keys<<<unsigned((A + 255) / 256), 256, 0, st>>>(active, A, t->N, t->inv, keys, slots);
    note_launch();
    int bits = 1;
    while ((int64_t(1) << bits) <= t->N) ++bits;
    T2_CHECK(radix_sort_u64_i32(keys, slots, A, st, bits));
    a.order = slots;
  }
  const void* fn = walk_kernel(t->nbp, kWalkWarps, false);
  const size_t smem = walk_smem(kWalkWarps, a.stack_ints, a.npix, a.max_depth);
  int per_sm = 0, sms = 0;
  T2_CHECK(config_walk_kernel(fn, kWalkWarps, smem, &per_sm, &sms));
  int64_t blocks = int64_t(sms) * per_sm;
  blocks = std::min<int64_t>(blocks, (A + kWalkWarps - 1) / kWalkWarps);
  blocks = std::max<int64_t>(blocks, 1);
  const size_t warps = size_t(blocks) * kWalkWarps;
  const size_t need = walk_buffer_bytes(warps, a.M);
  T2_CHECK(grow_buffer(&t->scratch, &t->scratch_bytes, need, st, "walk buffers"));
  place_walk_buffers(static_cast<char*>(t->scratch), warps, a.M, &a.srcU, &a.srcV, &a.srcT, &a.pixU);
  T2_CUDA(cudaMemsetAsync(t->counter, 0, sizeof(unsigned long long), st));
  void* args[] = {&a};
  T2_CUDA(cudaLaunchKernel(fn, dim3(unsigned(blocks)), dim3(kWalkWarps * 32), args, smem, st));
  note_launch();
  return TREVR2_OK;
}

// ---------------------------------------------------------------------------
// Complex source model tables (Sec. 2.7, Eq. srccomb), one depth at a time,
// deepest first, a thread per (cell, direction k).  A luminous cell's ray
// runs from its centre of luminosity along n_k to its box edge (length d);
// a leaf's optical depth is its bucket alpha times d.  A parent's ray ends
// on the plane through the end of its own ray, perpendicular to n_k: each
// luminous child's ray is clipped to that plane or extended to it through
// the sibling (the sibling's alpha for this direction pair over the
// extension's chord with its box), and L e^{-tau} = sum_i L_i e^{-tau_i'}
// per band, evaluated with the smallest tau_i' factored out so that opaque
// children do not underflow.
__global__ void k_csm_anti(int nside, int npix, const double* __restrict__ dirs64,
                           int* __restrict__ anti) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= npix) return;
  anti[k] = hp_vec2pix_f64(nside, -dirs64[3 * k], -dirs64[3 * k + 1], -dirs64[3 * k + 2]);
}

template <int NBP>
__global__ void k_csm_level(int64_t lb, int64_t le, int npix, int P,
                            const NodeW* __restrict__ nodes, const float4* __restrict__ csrc,
                            const float* __restrict__ Lnode, const float* __restrict__ alpha_leaf,
                            const float* __restrict__ alpha_tab, const float4* __restrict__ dirs,
                            float* __restrict__ csm_d, float* __restrict__ csm_tau) {
  const int64_t idx = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (idx >= (le - lb) * npix) return;
  const int64_t q = lb + idx / npix;
  const int k = int(idx % npix);
  const NodeW nd = nodes[q];
  if (!(nd.meta & kMetaHasL)) return;  // left at zero
  const float4 dn = dirs[k];
  const int pair = __float_as_int(dn.w);
  const float n[3] = {dn.x, dn.y, dn.z};
  float inv[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) inv[c] = n[c] != 0.0f ? 1.0f / n[c] : 0.0f;
  const float4 cq = csrc[q];
  const float xq[3] = {cq.x, cq.y, cq.z};
  float t0, t1;
  const float d = beam_chord(nd, xq, n, inv, INFINITY, t0, t1) ? t1 : 0.0f;
  csm_d[q * npix + k] = d;
  float* out = csm_tau + (q * npix + k) * NBP;
  if (nd.meta & kMetaLeaf) {
#pragma unroll
    for (int b = 0; b < NBP; ++b) out[b] = alpha_leaf[q * NBP + b] * d;
    return;
  }
  float tc[2][NBP], Lc[2][NBP];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int64_t i = nd.child + h;
    const NodeW ni = nodes[i];
#pragma unroll
    for (int b = 0; b < NBP; ++b) {
      tc[h][b] = 0.0f;
      Lc[h][b] = 0.0f;
    }
    if (!(ni.meta & kMetaHasL)) continue;
    const float4 ci = csrc[i];
    const float xi[3] = {ci.x, ci.y, ci.z};
    const float D = fmaxf((cq.x - ci.x) * n[0] + (cq.y - ci.y) * n[1] + (cq.z - ci.z) * n[2] + d,
                          0.0f);
    const float di = csm_d[i * npix + k];
    const int64_t sib = nd.child + (1 - h);
    const NodeW ns = nodes[sib];
    float ext = 0.0f;
    if (D > di) {
      float s0, s1;
      if (beam_chord(ns, xi, n, inv, INFINITY, s0, s1))
        ext = fmaxf(0.0f, fminf(s1, D) - fmaxf(s0, di));
    }
#pragma unroll
    for (int b = 0; b < NBP; ++b) {
      const float ti = csm_tau[(i * npix + k) * NBP + b];
      const float as = (ns.meta & kMetaLeaf) ? alpha_leaf[sib * NBP + b]
                                             : alpha_tab[(int64_t(ns.aux) * P + pair) * NBP + b];
      tc[h][b] = D <= di ? (di > 0.0f ? ti * (D / di) : 0.0f) : ti + as * ext;
      Lc[h][b] = Lnode[i * NBP + b];
    }
  }
#pragma unroll
  for (int b = 0; b < NBP; ++b) {
    const float Lq = Lnode[q * NBP + b];
    float m = INFINITY;
#pragma unroll
    for (int h = 0; h < 2; ++h)
      if (Lc[h][b] > 0.0f) m = fminf(m, tc[h][b]);
    if (!(Lq > 0.0f) || !(m < INFINITY)) {
      out[b] = 0.0f;
      continue;
    }
    float S = 0.0f;
#pragma unroll
    for (int h = 0; h < 2; ++h)
      if (Lc[h][b] > 0.0f) S += Lc[h][b] * expf(-(tc[h][b] - m));
    out[b] = m - logf(S / Lq);
  }
}

// The complex source model tables for this table's nside and averaging.
static int ensure_csm(Tree* t, Table* tb, cudaStream_t st) {
  if (tb->csm_tau) return TREVR2_OK;
  const int npix = 12 * tb->nside * tb->nside, P = npix / 2;
  const int64_t n = t->n_nodes;
  const size_t ntau = size_t(n) * npix * t->nbp, nd = size_t(n) * npix;
  // built in temporaries and kept by the table only when complete
  DeviceTemp<float> csm_tau(st), csm_d(st);
  DeviceTemp<int> csm_anti(st);
  T2_CHECK(device_alloc(reinterpret_cast<void**>(&csm_tau.p), ntau * sizeof(float), st,
                        "complex source model tables"));
  T2_CHECK(device_alloc(reinterpret_cast<void**>(&csm_d.p), nd * sizeof(float), st,
                        "complex source model tables"));
  T2_CHECK(device_alloc(reinterpret_cast<void**>(&csm_anti.p), npix * sizeof(int), st,
                        "complex source model tables"));
  T2_CUDA(cudaMemsetAsync(csm_tau.p, 0, ntau * sizeof(float), st));
  T2_CUDA(cudaMemsetAsync(csm_d.p, 0, nd * sizeof(float), st));
  k_csm_anti<<<(npix + 127) / 128, 128, 0, st>>>(tb->nside, npix, tb->dirs64, csm_anti.p);
  note_launch();
  for (int d = t->max_depth; d >= 0; --d) {
    const int64_t lb = t->level_begin[d], le = t->level_begin[d + 1];
    const int64_t work = (le - lb) * npix;
    if (work <= 0) continue;
    const unsigned blocks = unsigned((work + 255) / 256);
    switch (t->nbp) {
      case 1: k_csm_level<1><<<blocks, 256, 0, st>>>(lb, le, npix, P, t->nodes, t->csrc, t->Lnode, t->alpha_leaf, tb->alpha, tb->dirs, csm_d.p, csm_tau.p); break;
      case 2: k_csm_level<2><<<blocks, 256, 0, st>>>(lb, le, npix, P, t->nodes, t->csrc, t->Lnode, t->alpha_leaf, tb->alpha, tb->dirs, csm_d.p, csm_tau.p); break;
      default: k_csm_level<4><<<blocks, 256, 0, st>>>(lb, le, npix, P, t->nodes, t->csrc, t->Lnode, t->alpha_leaf, tb->alpha, tb->dirs, csm_d.p, csm_tau.p); break;
    }
    note_launch();
  }
  T2_CUDA(cudaGetLastError());
  tb->csm_tau = csm_tau.p;
  tb->csm_d = csm_d.p;
  tb->csm_anti = csm_anti.p;
  csm_tau.p = csm_d.p = nullptr;
  csm_anti.p = nullptr;
  return TREVR2_OK;
}

template <int NBP>
static const void* bucket_kernel_nbp(bool pp, bool csm) {
  if (csm)
    return pp ? reinterpret_cast<const void*>(&k_walk_bucket<NBP, kWalkWarps, true, true>)
              : reinterpret_cast<const void*>(&k_walk_bucket<NBP, kWalkWarps, false, true>);
  return pp ? reinterpret_cast<const void*>(&k_walk_bucket<NBP, kWalkWarps, true, false>)
            : reinterpret_cast<const void*>(&k_walk_bucket<NBP, kWalkWarps, false, false>);
}

// p-p particles one warp holds for a bucket (TREVR2_PP); a bucket whose
// sphere holds more is reported (EUNSUPPORTED).
constexpr int kPPCapacity = 4096;

template <int NBP>
static const void* bucket_batched_kernel_nbp(bool pp, bool csm) {
  if (csm)
    return pp ? reinterpret_cast<const void*>(&k_walk_bucket_batched<NBP, kWalkWarps, true, true>)
              : reinterpret_cast<const void*>(&k_walk_bucket_batched<NBP, kWalkWarps, false, true>);
  return pp ? reinterpret_cast<const void*>(&k_walk_bucket_batched<NBP, kWalkWarps, true, false>)
            : reinterpret_cast<const void*>(&k_walk_bucket_batched<NBP, kWalkWarps, false, false>);
}

static const void* bucket_batched_kernel(int nbp, bool pp, bool csm) {
  return nbp == 1 ? bucket_batched_kernel_nbp<1>(pp, csm)
       : nbp == 2 ? bucket_batched_kernel_nbp<2>(pp, csm)
                  : bucket_batched_kernel_nbp<4>(pp, csm);
}

// TREVR2_BUCKET: receivers in Morton order, the leaf of each, one warp per
// bucket.
static int launch_walk_bucket(Tree* t, Table* tb, const int64_t* active, int64_t A, int nside,
                              float theta, const int* bsel, int nbsel, uint32_t flags, float* J,
                              const double* target, cudaStream_t st) {
  WalkArgs a;
  // the walk from the bucket centre takes no receiver flags; they go to bk
  fill_walk_args(t, tb, nside, theta, bsel, nbsel, flags & ~(TREVR2_SOFT | TREVR2_THICK),
                 kSrcCapacity, &a);
  a.active = active;
  a.A = A;
  a.J = J;
  const size_t need_order = size_t(A) * (sizeof(uint64_t) + 2 * sizeof(int));
  T2_CHECK(grow_buffer(&t->order_buf, &t->order_bytes, need_order, st, "receiver order"));
  uint64_t* keys = static_cast<uint64_t*>(t->order_buf);
  int* slots = reinterpret_cast<int*>(keys + A);
  int* leaf = slots + A;
  const unsigned gb = unsigned((A + 255) / 256);
  k_order_keys<<<gb, 256, 0, st>>>(active, A, t->N, t->inv, keys, slots);
  note_launch();
  if (A > 1) {
    int bits = 1;
    while ((int64_t(1) << bits) <= t->N) ++bits;
    T2_CHECK(radix_sort_u64_i32(keys, slots, A, st, bits));
  }
  k_bucket_leaf<<<gb, 256, 0, st>>>(t->child, t->first, keys, A, t->N, leaf);
  note_launch();
  a.order = slots;
  if (flags & TREVR2_CSM) {
    T2_CHECK(ensure_csm(t, tb, st));
    a.csm_tau = tb->csm_tau;
    a.csm_d = tb->csm_d;
    a.csm_anti = tb->csm_anti;
  }
  BucketArgs bk;
  std::memset(&bk, 0, sizeof(bk));
  bk.keys = keys;
  bk.leaf = leaf;
  bk.rflags = flags & (TREVR2_SOFT | TREVR2_THICK);
  bk.pp = (flags & TREVR2_PP) != 0;
  bk.pp_cap = bk.pp ? kPPCapacity : 0;
  bk.beam = std::sqrt(4.0 * M_PI / double(a.npix));
  bk.mass = t->mass;
  bk.directed = target != nullptr;
  for (int c = 0; c < 3; ++c) bk.target[c] = target ? (target[c] - t->lo[c]) / t->size : 0.0;
  const bool csm = (flags & TREVR2_CSM) != 0;
  const void* fn = t->nbp == 1 ? bucket_kernel_nbp<1>(bk.pp, csm)
                 : t->nbp == 2 ? bucket_kernel_nbp<2>(bk.pp, csm)
                               : bucket_kernel_nbp<4>(bk.pp, csm);
  const size_t smem = walk_smem(kWalkWarps, a.stack_ints, a.npix, a.max_depth);
  int per_sm = 0, sms = 0;
  T2_CHECK(config_walk_kernel(fn, kWalkWarps, smem, &per_sm, &sms));
  int64_t blocks = int64_t(sms) * per_sm;
  blocks = std::min<int64_t>(blocks, (A + kWalkWarps - 1) / kWalkWarps);
  blocks = std::max<int64_t>(blocks, 1);
  const size_t warps = size_t(blocks) * kWalkWarps;
  const size_t wb = (walk_buffer_bytes(warps, a.M) + 255) & ~size_t(255);
  const size_t ob = (warps * kOriginWords * sizeof(double) + 255) & ~size_t(255);
  const size_t pb = warps * size_t(bk.pp_cap) *
                    (4 * sizeof(float4) + sizeof(int) + kCubeCells / 32 * sizeof(uint32_t));
  const size_t need = wb + ob + pb;
  T2_CHECK(grow_buffer(&t->scratch, &t->scratch_bytes, need, st, "walk buffers"));
  place_walk_buffers(static_cast<char*>(t->scratch), warps, a.M, &a.srcU, &a.srcV, &a.srcT, &a.pixU);
  a.origin64 = reinterpret_cast<double*>(static_cast<char*>(t->scratch) + wb);
  if (bk.pp) {
    char* pp = static_cast<char*>(t->scratch) + wb + ob;
    bk.pp_xh = reinterpret_cast<float4*>(pp);
    bk.pp_kc = bk.pp_xh + warps * bk.pp_cap;
    bk.pp_w = bk.pp_kc + warps * bk.pp_cap;
    bk.pp_u = bk.pp_w + warps * bk.pp_cap;
    bk.pp_si = reinterpret_cast<int*>(bk.pp_u + warps * bk.pp_cap);
    bk.pp_mask = reinterpret_cast<uint32_t*>(bk.pp_si + warps * bk.pp_cap);
  }
  T2_CUDA(cudaMemsetAsync(t->counter, 0, sizeof(unsigned long long), st));
  void* args[] = {&a, &bk};
  T2_CUDA(cudaLaunchKernel(fn, dim3(unsigned(blocks)), dim3(kWalkWarps * 32), args, smem, st));
  note_launch();
  return TREVR2_OK;
}

int read_status(Tree* t, cudaStream_t st) {
  uint32_t s = 0;
  T2_CUDA(cudaMemcpyAsync(&s, t->status, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
  T2_CUDA(cudaStreamSynchronize(st));
  if (s == 0) return TREVR2_OK;
  T2_CUDA(cudaMemsetAsync(t->status, 0, sizeof(uint32_t), st));
  if (s & kStatusBadActive) {
    set_error("trevr2_J: an active index lies outside [0, N) (its row is NaN)");
    return TREVR2_EINVAL;
  }
  if (s & kStatusStackOverflow) {
    set_error("trevr2_J: internal traversal stack overflow");
    return TREVR2_EINTERNAL;
  }
  if (s & kStatusPPOverflow) {
    set_error("trevr2_J: a bucket's p-p sphere holds more than %d particles (TREVR2_PP)",
              kPPCapacity);
    return TREVR2_EUNSUPPORTED;
  }
  set_error("trevr2: device status 0x%x", s);
  return TREVR2_EINTERNAL;
}

}  // namespace trevr2

using namespace trevr2;

// trevr2_J and trevr2_J_directed (target != NULL).
static int J_impl(trevr2_tree* tree, const int64_t* active, int64_t A, int nside, float theta,
                  const int* bands, int nbsel, uint32_t flags, const double* target, float* J,
                  void* stream) {
  clear_error();
  if (!tree) {
    set_error("trevr2_J: tree is NULL");
    return TREVR2_EINVAL;
  }
  if (target) {
    if (!(flags & TREVR2_BUCKET)) {
      set_error("trevr2_J_directed: directed rays need TREVR2_BUCKET");
      return TREVR2_EINVAL;
    }
    for (int c = 0; c < 3; ++c) {
      if (!std::isfinite(target[c])) {
        set_error("trevr2_J_directed: the target is not finite");
        return TREVR2_EINVAL;
      }
    }
  }
  Tree* t = reinterpret_cast<Tree*>(tree);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  t->last_stream = st;
  if (A < 0 || (A > 0 && (!active || !J))) {
    set_error("trevr2_J: A < 0 or NULL active/J");
    return TREVR2_EINVAL;
  }
  if (!valid_nside(nside)) {
    set_error("trevr2_J: nside %d is not a power of two in [1, %d]", nside, TREVR2_MAX_NSIDE);
    return nside > TREVR2_MAX_NSIDE ? TREVR2_EUNSUPPORTED : TREVR2_EINVAL;
  }
  if (!(theta > 0.0f) || !std::isfinite(theta)) {
    set_error("trevr2_J: theta must be positive and finite");
    return TREVR2_EINVAL;
  }
  if (flags & ~(TREVR2_SOFT | TREVR2_THICK | TREVR2_LINEAR | TREVR2_ASYNC | TREVR2_BUCKET |
                TREVR2_PP | TREVR2_CSM)) {
    set_error("trevr2_J: unknown flag bits 0x%x", flags);
    return TREVR2_EINVAL;
  }
  if ((flags & (TREVR2_PP | TREVR2_CSM)) && !(flags & TREVR2_BUCKET)) {
    set_error("trevr2_J: TREVR2_PP and TREVR2_CSM need TREVR2_BUCKET");
    return TREVR2_EINVAL;
  }
  int bsel[TREVR2_MAX_BANDS];
  if (bands) {
    if (nbsel < 1 || nbsel > t->nb) {
      set_error("trevr2_J: nbsel = %d outside [1, %d]", nbsel, t->nb);
      return TREVR2_EINVAL;
    }
    for (int b = 0; b < nbsel; ++b) {
      if (bands[b] < 0 || bands[b] >= t->nb) {
        set_error("trevr2_J: band index %d outside [0, %d)", bands[b], t->nb);
        return TREVR2_EINVAL;
      }
      bsel[b] = bands[b];
    }
  } else {
    nbsel = t->nb;
    for (int b = 0; b < nbsel; ++b) bsel[b] = b;
  }
  if (A == 0) return TREVR2_OK;
  Table* tb = nullptr;
  T2_CHECK(ensure_table(t, nside, st, &tb, (flags & TREVR2_LINEAR) != 0));
  if (flags & TREVR2_BUCKET)
    T2_CHECK(launch_walk_bucket(t, tb, active, A, nside, theta, bsel, nbsel, flags, J, target,
                                st));
  else
    T2_CHECK(launch_walk(t, tb, active, A, nside, theta, bsel, nbsel, flags, J, st));
  if (flags & TREVR2_ASYNC) return TREVR2_OK;
  return read_status(t, st);
}

extern "C" int trevr2_J(trevr2_tree* tree, const int64_t* active, int64_t A, int nside, float theta,
                        const int* bands, int nbsel, uint32_t flags, float* J, void* stream) {
  return J_impl(tree, active, A, nside, theta, bands, nbsel, flags, nullptr, J, stream);
}

extern "C" int trevr2_J_directed(trevr2_tree* tree, const int64_t* active, int64_t A, int nside,
                                 float theta, const int* bands, int nbsel, uint32_t flags,
                                 const double* target, float* J, void* stream) {
  if (!target) {
    clear_error();
    set_error("trevr2_J_directed: target is NULL");
    return TREVR2_EINVAL;
  }
  return J_impl(tree, active, A, nside, theta, bands, nbsel, flags, target, J, stream);
}

// ---------------------------------------------------------------------------
// Batches: many active subsets over several trees in one persistent launch.
namespace trevr2 {

struct Batch {
  std::vector<Tree*> trees;
  int nside = 0;
  int nsub = 0;
  int64_t total = 0;
  int nbp = 1;
  int64_t* d_offsets = nullptr;
  int* d_tree_of = nullptr;
  unsigned long long* counter = nullptr;
  void* scratch = nullptr;
  size_t scratch_bytes = 0;
  void* dedup = nullptr;     // keys, rows, scan, distinct keys, their J, sort workspace
  void* sort_ws = nullptr;
  int* scan_ws = nullptr;
  int key_bits = 64;
  int warps = kWalkWarps;  // chosen launch shape
  int M = kSrcCapacity;    // chosen source staging depth
  const void* fn = nullptr;  // kernel, shared memory and grid of that shape
  size_t smem = 0;
  int64_t blocks = 0;
  bool ready = false;        // the shape covers every row (false after a failed autotune)
  cudaStream_t last_stream = nullptr;
  // per-bucket plans (TREVR2_BUCKET, with TREVR2_PP / TREVR2_CSM)
  bool bucket = false;
  bool pp = false;
  bool csm = false;
  BucketBatchArgs bb;
  BatchArgs args;
};

// Selects the launch shape (warps, M) for the first `limit` rows: kernel,
// grid and walk buffers (grown if needed).  Nothing changes unless it
// succeeds: a larger buffer is allocated before the old one is released.
static int batch_select(Batch* b, int warps, int M, int64_t limit, cudaStream_t st) {
  const void* fn = b->bucket ? bucket_batched_kernel(b->nbp, b->pp, b->csm)
                             : walk_kernel(b->nbp, warps, true);
  const size_t smem = walk_smem(warps, b->args.stack_ints, b->args.npix, b->args.max_depth);
  int per_sm = 0, sms = 0;
  T2_CHECK(config_walk_kernel(fn, warps, smem, &per_sm, &sms));
  int64_t g = int64_t(sms) * per_sm;
  g = std::min<int64_t>(g, (limit + warps - 1) / warps);
  const int64_t blocks = std::max<int64_t>(g, 1);
  const size_t nw = size_t(blocks) * warps;
  // per-bucket plans: the warps' FP64 origin slots and p-p particle arrays
  const size_t wb = (walk_buffer_bytes(nw, M) + 255) & ~size_t(255);
  const size_t ob = b->bucket ? (nw * kOriginWords * sizeof(double) + 255) & ~size_t(255) : 0;
  const size_t pp_cap = b->pp ? kPPCapacity : 0;
  const size_t pb = nw * pp_cap *
                    (4 * sizeof(float4) + sizeof(int) + kCubeCells / 32 * sizeof(uint32_t));
  const size_t need = wb + ob + pb;
  if (b->scratch_bytes < need) {
    void* fresh = nullptr;
    T2_CHECK(device_alloc(&fresh, need, st, "batch walk buffers"));
    if (b->scratch) cudaFreeAsync(b->scratch, st);
    b->scratch = fresh;
    b->scratch_bytes = need;
  }
  place_walk_buffers(static_cast<char*>(b->scratch), nw, M, &b->args.srcU, &b->args.srcV,
                     &b->args.srcT, &b->args.pixU);
  b->args.M = M;
  for (size_t i = 0; i < b->trees.size(); ++i) b->args.tree[i].M = M;
  if (b->bucket) {
    char* base = static_cast<char*>(b->scratch);
    double* origin = reinterpret_cast<double*>(base + wb);
    float4* pp = reinterpret_cast<float4*>(base + wb + ob);
    for (size_t i = 0; i < b->trees.size(); ++i) {
      b->args.tree[i].origin64 = origin;
      BucketArgs& bk = b->bb.tree[i];
      bk.pp_cap = int(pp_cap);
      bk.pp_xh = b->pp ? pp : nullptr;
      bk.pp_kc = b->pp ? pp + nw * pp_cap : nullptr;
      bk.pp_w = b->pp ? pp + 2 * nw * pp_cap : nullptr;
      bk.pp_u = b->pp ? pp + 3 * nw * pp_cap : nullptr;
      bk.pp_si = b->pp ? reinterpret_cast<int*>(pp + 4 * nw * pp_cap) : nullptr;
      bk.pp_mask = b->pp ? reinterpret_cast<uint32_t*>(reinterpret_cast<int*>(pp + 4 * nw * pp_cap) +
                                                      nw * pp_cap)
                         : nullptr;
    }
  }
  b->fn = fn;
  b->smem = smem;
  b->blocks = blocks;
  b->warps = warps;
  b->M = M;
  b->args.total = limit;
  b->ready = limit == b->total;
  return TREVR2_OK;
}

// Enqueues the run in the selected shape (keys, sort, distinct keys, walk,
// scatter) with no allocation, synchronisation or attribute call, so that it
// can be recorded into a CUDA graph.
static int batch_enqueue(Batch* b, const int64_t* active, float* J, cudaStream_t st) {
  b->args.active = active;
  b->args.J = J;
  const int64_t R = b->args.total;
  if (R <= 0) return TREVR2_OK;
  const unsigned g = unsigned((R + 255) / 256);
  T2_CUDA(cudaMemsetAsync(b->counter, 0, sizeof(unsigned long long), st));
  k_batch_keys<<<g, 256, 0, st>>>(b->args); note_launch();
  T2_CHECK(radix_sort_u64_i32(b->args.keys, b->args.rows, R, st, b->key_bits, b->sort_ws));
  k_batch_first<<<g, 256, 0, st>>>(b->args); note_launch();
  T2_CHECK(scan_exclusive_i32(b->args.first_scan, R, b->args.n_distinct, st, b->scan_ws));
  k_batch_distinct<<<g, 256, 0, st>>>(b->args); note_launch();
  if (b->bucket) {
    k_batch_leaf<<<g, 256, 0, st>>>(b->args, b->bb);
    note_launch();
  }
  k_batch_tree_range<<<1, 64, 0, st>>>(b->args); note_launch();
  // one walk launch per tree, each over that tree's distinct keys
  BatchSlice sl;
  sl.ukeys = b->args.ukeys;
  sl.ubkey = b->args.ubkey;
  sl.tree_range = b->args.tree_range;
  sl.Ju = b->args.Ju;
  sl.key_shift = b->args.key_shift;
  sl.nbsel = b->args.nbsel;
  sl.srcU = b->args.srcU;
  sl.pixU = b->args.pixU;
  sl.srcV = b->args.srcV;
  sl.srcT = b->args.srcT;
  sl.counter = b->counter;
  for (int t = 0; t < b->args.ntrees; ++t) {
    sl.t = t;
    T2_CUDA(cudaMemsetAsync(b->counter, 0, sizeof(unsigned long long), st));
    if (b->bucket) {
      void* argv[] = {&b->args.tree[t], &b->bb.tree[t], &sl};
      T2_CUDA(cudaLaunchKernel(b->fn, dim3(unsigned(b->blocks)), dim3(b->warps * 32), argv,
                               b->smem, st));
    } else {
      void* argv[] = {&b->args.tree[t], &sl};
      T2_CUDA(cudaLaunchKernel(b->fn, dim3(unsigned(b->blocks)), dim3(b->warps * 32), argv,
                               b->smem, st));
    }
    note_launch();
  }
  k_batch_scatter<<<g, 256, 0, st>>>(b->args); note_launch();
  T2_CUDA(cudaGetLastError());
  return TREVR2_OK;
}

static void free_batch(Batch* b, cudaStream_t st) {
  dfree(b->d_offsets, st);
  dfree(b->d_tree_of, st);
  dfree(b->counter, st);
  if (b->scratch) cudaFreeAsync(b->scratch, st);
  b->scratch = nullptr;
  if (b->dedup) cudaFreeAsync(b->dedup, st);
  b->dedup = nullptr;
}

}  // namespace trevr2

extern "C" int trevr2_batch_create(trevr2_tree* const* trees, int ntrees, const int64_t* offsets,
                                   const int* tree_of, int nsub, int nside, float theta,
                                   uint32_t flags, void* stream, trevr2_batch** out) {
  clear_error();
  if (!out) {
    set_error("trevr2_batch_create: out is NULL");
    return TREVR2_EINVAL;
  }
  *out = nullptr;
  if (!trees || ntrees < 1 || nsub < 0 || (nsub > 0 && (!offsets || !tree_of))) {
    set_error("trevr2_batch_create: NULL arrays, ntrees < 1 or nsub < 0");
    return TREVR2_EINVAL;
  }
  if (ntrees > kMaxBatchTrees) {
    set_error("trevr2_batch_create: at most %d trees per batch", kMaxBatchTrees);
    return TREVR2_EUNSUPPORTED;
  }
  if (!valid_nside(nside)) {
    set_error("trevr2_batch_create: nside %d is not a power of two in [1, %d]", nside,
              TREVR2_MAX_NSIDE);
    return nside > TREVR2_MAX_NSIDE ? TREVR2_EUNSUPPORTED : TREVR2_EINVAL;
  }
  if (!(theta > 0.0f) || !std::isfinite(theta) ||
      (flags & ~(TREVR2_SOFT | TREVR2_THICK | TREVR2_LINEAR | TREVR2_ASYNC | TREVR2_BUCKET |
                 TREVR2_PP | TREVR2_CSM))) {
    set_error("trevr2_batch_create: theta must be positive and finite, flags "
              "SOFT|THICK|LINEAR|BUCKET|PP|CSM|ASYNC");
    return TREVR2_EINVAL;
  }
  if ((flags & (TREVR2_PP | TREVR2_CSM)) && !(flags & TREVR2_BUCKET)) {
    set_error("trevr2_batch_create: TREVR2_PP and TREVR2_CSM need TREVR2_BUCKET");
    return TREVR2_EINVAL;
  }
  const int nb = reinterpret_cast<Tree*>(trees[0])->nb;
  for (int i = 0; i < ntrees; ++i) {
    if (!trees[i] || reinterpret_cast<Tree*>(trees[i])->nb != nb) {
      set_error("trevr2_batch_create: tree %d is NULL or has a different band count", i);
      return TREVR2_EINVAL;
    }
  }
  if (nsub > 0 && offsets[0] != 0) {
    set_error("trevr2_batch_create: offsets[0] must be 0");
    return TREVR2_EINVAL;
  }
  if (nsub > 0 && offsets[nsub] >= (int64_t(1) << 31)) {
    set_error("trevr2_batch_create: at most 2^31 - 1 rows per batch");
    return TREVR2_EUNSUPPORTED;
  }
  for (int s = 0; s < nsub; ++s) {
    if (offsets[s + 1] < offsets[s] || tree_of[s] < 0 || tree_of[s] >= ntrees) {
      set_error("trevr2_batch_create: offsets must not decrease and tree_of must index the trees "
                "(subset %d)", s);
      return TREVR2_EINVAL;
    }
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Batch* b = new (std::nothrow) Batch();
  if (!b) {
    set_error("trevr2_batch_create: host allocation failed");
    return TREVR2_ENOMEM;
  }
  auto fail = [&](int rc) {
    std::string msg = trevr2_last_error();
    free_batch(b, st);
    delete b;
    set_error("%s", msg.c_str());
    return rc;
  };
  b->nside = nside;
  b->nsub = nsub;
  b->total = nsub > 0 ? offsets[nsub] : 0;
  b->nbp = nbp_of(nb);
  b->last_stream = st;
  b->bucket = (flags & TREVR2_BUCKET) != 0;
  b->pp = (flags & TREVR2_PP) != 0;
  b->csm = (flags & TREVR2_CSM) != 0;
  std::memset(&b->args, 0, sizeof(BatchArgs));
  std::memset(&b->bb, 0, sizeof(BucketBatchArgs));
  int max_depth = 0;
  int bsel[TREVR2_MAX_BANDS];
  for (int k = 0; k < nb; ++k) bsel[k] = k;
  for (int i = 0; i < ntrees; ++i) {
    Tree* t = reinterpret_cast<Tree*>(trees[i]);
    t->last_stream = st;
    b->trees.push_back(t);
    max_depth = std::max(max_depth, t->max_depth);
    Table* tb = nullptr;
    int rc = ensure_table(t, nside, st, &tb, (flags & TREVR2_LINEAR) != 0);
    if (rc) return fail(rc);
    if (!b->bucket) {
      fill_walk_args(t, tb, nside, theta, bsel, nb, flags & ~TREVR2_ASYNC, kSrcCapacity,
                     &b->args.tree[i]);
      continue;
    }
    // the walk from the bucket centre takes no receiver flags; they go to the
    // bucket arguments (as in trevr2_J with TREVR2_BUCKET)
    WalkArgs& a = b->args.tree[i];
    fill_walk_args(t, tb, nside, theta, bsel, nb,
                   flags & ~(TREVR2_SOFT | TREVR2_THICK | TREVR2_ASYNC), kSrcCapacity, &a);
    if (b->csm) {
      rc = ensure_csm(t, tb, st);
      if (rc) return fail(rc);
      a.csm_tau = tb->csm_tau;
      a.csm_d = tb->csm_d;
      a.csm_anti = tb->csm_anti;
    }
    BucketArgs& bk = b->bb.tree[i];
    bk.rflags = flags & (TREVR2_SOFT | TREVR2_THICK);
    bk.pp = b->pp ? 1 : 0;
    bk.beam = std::sqrt(4.0 * M_PI / double(12 * nside * nside));
    bk.mass = t->mass;
    bk.directed = 0;
    b->bb.child[i] = t->child;
    b->bb.first[i] = t->first;
  }
  // one shared-memory layout for all trees: the deepest one's
  for (int i = 0; i < ntrees; ++i) {
    b->args.tree[i].max_depth = max_depth;
    b->args.tree[i].stack_ints = 64 * (max_depth + 2);
    b->args.tree[i].src_stack_cap = b->args.tree[i].stack_ints;
    if (const int cap = debug_source_stack_cap())
      b->args.tree[i].src_stack_cap = std::min(cap, b->args.tree[i].stack_ints);
  }
  b->args.max_depth = max_depth;
  b->args.stack_ints = 64 * (max_depth + 2);
  b->args.npix = 12 * nside * nside;
  b->args.nbsel = nb;
  b->args.nsub = nsub;
  b->args.ntrees = ntrees;
  int64_t maxN = 1;
  for (Tree* t : b->trees) maxN = std::max<int64_t>(maxN, t->N);
  int shift = 1;
  while ((int64_t(1) << shift) < maxN) ++shift;
  b->args.key_shift = shift;
  b->key_bits = shift + 6;  // trees and the invalid marker: at most 33 values
  int rc = dalloc(&b->d_offsets, size_t(nsub) + 1, st);
  if (!rc) rc = dalloc(&b->d_tree_of, size_t(std::max(nsub, 1)), st);
  if (!rc) rc = dalloc(&b->counter, 1, st);
  if (rc) return fail(rc);
  if (b->total > 0) {
    // deduplication buffers for all rows, allocated once
    auto up = [](size_t v) { return (v + 255) & ~size_t(255); };
    const size_t R = size_t(b->total);
    const size_t bk = up(8 * R), br = up(4 * R), bu = up(4 * R * nb);
    const size_t bsort = up(radix_ws_bytes(int64_t(R))), bscan = up(4 * scan_ws_ints(int64_t(R)));
    const size_t bbuck = b->bucket ? bk * 2 + br : 0;  // usi, ubkey, uorder
    const size_t brange = up(sizeof(int) * (kMaxBatchTrees + 1));
    const size_t bytes = bk * 2 + br * 2 + bu + 256 + bsort + bscan + bbuck + brange;
    rc = device_alloc(&b->dedup, bytes, st, "batch deduplication buffers");
    if (rc) return fail(rc);
    char* p = static_cast<char*>(b->dedup);
    b->args.keys = reinterpret_cast<uint64_t*>(p); p += bk;
    b->args.ukeys = reinterpret_cast<uint64_t*>(p); p += bk;
    b->args.rows = reinterpret_cast<int*>(p); p += br;
    b->args.first_scan = reinterpret_cast<int*>(p); p += br;
    b->args.Ju = reinterpret_cast<float*>(p); p += bu;
    b->args.n_distinct = reinterpret_cast<int*>(p); p += 256;
    b->sort_ws = p; p += bsort;
    b->scan_ws = reinterpret_cast<int*>(p); p += bscan;
    b->args.tree_range = reinterpret_cast<int*>(p); p += brange;
    if (b->bucket) {
      b->args.usi = reinterpret_cast<uint64_t*>(p); p += bk;
      b->args.ubkey = reinterpret_cast<uint64_t*>(p); p += bk;
      b->args.uorder = reinterpret_cast<int*>(p);
      // the per-bucket walk writes each distinct key's row of Ju through its
      // order (the identity)
      for (int i = 0; i < ntrees; ++i) {
        b->args.tree[i].J = b->args.Ju;
        b->args.tree[i].order = b->args.uorder;
        b->bb.tree[i].keys = b->args.usi;
      }
    }
  }
  if (nsub > 0) {
    cudaError_t e = cudaMemcpyAsync(b->d_offsets, offsets, (size_t(nsub) + 1) * sizeof(int64_t),
                                    cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(b->d_tree_of, tree_of, size_t(nsub) * sizeof(int), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(cuda_fail(e, "cudaMemcpyAsync(batch metadata)"));
  }
  b->args.offsets = b->d_offsets;
  b->args.tree_of = b->d_tree_of;
  b->args.counter = b->counter;
  // the default shape and its buffers, so that run() never allocates
  rc = batch_select(b, kWalkWarps, kSrcCapacity, b->total, st);
  if (rc) return fail(rc);
  *out = reinterpret_cast<trevr2_batch*>(b);
  return TREVR2_OK;
}

extern "C" int trevr2_batch_run(trevr2_batch* batch, const int64_t* active, float* J, void* stream) {
  clear_error();
  if (!batch) {
    set_error("trevr2_batch_run: batch is NULL");
    return TREVR2_EINVAL;
  }
  Batch* b = reinterpret_cast<Batch*>(batch);
  if (b->total > 0 && (!active || !J)) {
    set_error("trevr2_batch_run: NULL active or J");
    return TREVR2_EINVAL;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  b->last_stream = st;
  if (b->total == 0) return TREVR2_OK;
  if (!b->ready) {
    set_error("trevr2_batch_run: the plan has no launch shape for all its rows (an earlier "
              "trevr2_batch_autotune failed); call trevr2_batch_autotune again or create a "
              "new plan");
    return TREVR2_EINVAL;
  }
  return batch_enqueue(b, active, J, st);
}

extern "C" int trevr2_batch_autotune(trevr2_batch* batch, const int64_t* active, float* J,
                                     void* stream, int* warps_out, int* staging_out) {
  clear_error();
  if (!batch) {
    set_error("trevr2_batch_autotune: batch is NULL");
    return TREVR2_EINVAL;
  }
  Batch* b = reinterpret_cast<Batch*>(batch);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  b->last_stream = st;
  if (b->total > 0 && (!active || !J)) {
    set_error("trevr2_batch_autotune: NULL active or J");
    return TREVR2_EINVAL;
  }
  if (b->total > 0) {
    // time each (warps per block, source staging depth) on a prefix of the
    // work and keep the fastest
    const int64_t limit = std::min<int64_t>(b->total, 65536);
    // the per-bucket walk is compiled for one block shape
    const int cand_w[2] = {4, 8};
    const int n_w = b->bucket ? 1 : 2;
    const int cand_m[3] = {512, 1024, 2048};
    cudaEvent_t e0, e1;
    T2_CUDA(cudaEventCreate(&e0));
    T2_CUDA(cudaEventCreate(&e1));
    float best = INFINITY;
    int bw = b->warps, bm = b->M;
    for (int iw = 0; iw < n_w; ++iw)
      for (int m : cand_m) {
        const int w = cand_w[iw];
        int rc = batch_select(b, w, m, limit, st);
        if (!rc) rc = batch_enqueue(b, active, J, st);  // warm-up
        if (!rc) {
          cudaError_t e = cudaEventRecord(e0, st);
          if (e == cudaSuccess) rc = batch_enqueue(b, active, J, st);
          if (e == cudaSuccess && !rc) e = cudaEventRecord(e1, st);
          if (e != cudaSuccess) rc = cuda_fail(e, "cudaEventRecord");
        }
        if (rc) {
          cudaEventDestroy(e0);
          cudaEventDestroy(e1);
          return rc;
        }
        T2_CUDA(cudaEventSynchronize(e1));
        float ms = 0.0f;
        T2_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        if (ms < best) {
          best = ms;
          bw = w;
          bm = m;
        }
      }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    // the chosen shape and its buffers at full size
    T2_CHECK(batch_select(b, bw, bm, b->total, st));
    T2_CUDA(cudaStreamSynchronize(st));
  }
  if (warps_out) *warps_out = b->warps;
  if (staging_out) *staging_out = b->M;
  return TREVR2_OK;
}

extern "C" int trevr2_batch_status(trevr2_batch* batch, void* stream) {
  clear_error();
  if (!batch) {
    set_error("trevr2_batch_status: batch is NULL");
    return TREVR2_EINVAL;
  }
  Batch* b = reinterpret_cast<Batch*>(batch);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int rc = TREVR2_OK;
  for (Tree* t : b->trees) {
    const int r = read_status(t, st);
    if (r != TREVR2_OK && rc == TREVR2_OK) rc = r;
  }
  return rc;
}

extern "C" int trevr2_batch_free(trevr2_batch* batch) {
  clear_error();
  if (!batch) return TREVR2_OK;
  Batch* b = reinterpret_cast<Batch*>(batch);
  free_batch(b, b->last_stream);
  delete b;
  return TREVR2_OK;
}

extern "C" int trevr2_J_batched(trevr2_tree* const* trees, int ntrees, const int64_t* active,
                                const int64_t* offsets, const int* tree_of, int nsub, int nside,
                                float theta, uint32_t flags, float* J, void* stream) {
  trevr2_batch* b = nullptr;
  T2_CHECK(trevr2_batch_create(trees, ntrees, offsets, tree_of, nsub, nside, theta, flags, stream, &b));
  int rc = trevr2_batch_run(b, active, J, stream);
  if (rc == TREVR2_OK && !(flags & TREVR2_ASYNC)) rc = trevr2_batch_status(b, stream);
  std::string msg = trevr2_last_error();
  trevr2_batch_free(b);
  if (rc != TREVR2_OK) set_error("%s", msg.c_str());
  return rc;
}

extern "C" int trevr2_kernel_binary_version(int* version) {
  clear_error();
  if (!version) {
    set_error("trevr2_kernel_binary_version: version is NULL");
    return TREVR2_EINVAL;
  }
  cudaFuncAttributes attr;
  T2_CUDA(cudaFuncGetAttributes(&attr, reinterpret_cast<const void*>(&k_walk<4, kWalkWarps>)));
  *version = attr.binaryVersion;
  return TREVR2_OK;
}

extern "C" int trevr2_status(trevr2_tree* tree, void* stream) {
  clear_error();
  if (!tree) {
    set_error("trevr2_status: tree is NULL");
    return TREVR2_EINVAL;
  }
  return read_status(reinterpret_cast<Tree*>(tree), static_cast<cudaStream_t>(stream));
}

extern "C" int trevr2_prepare(trevr2_tree* tree, int nside, void* stream) {
  clear_error();
  if (!tree) {
    set_error("trevr2_prepare: tree is NULL");
    return TREVR2_EINVAL;
  }
  if (!valid_nside(nside)) {
    set_error("trevr2_prepare: nside %d is not a power of two in [1, %d]", nside, TREVR2_MAX_NSIDE);
    return nside > TREVR2_MAX_NSIDE ? TREVR2_EUNSUPPORTED : TREVR2_EINVAL;
  }
  Tree* t = reinterpret_cast<Tree*>(tree);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  t->last_stream = st;
  Table* tb = nullptr;
  return ensure_table(t, nside, st, &tb);
}

// ---------------------------------------------------------------------------
// Allocation-free variant of trevr2_J.
//
// Some host codes cannot let a library call cudaMalloc: they own every byte
// of device memory through their own arena or a fixed memory budget, or they
// call in from a context where a device allocation could block or fail.  For
// them the walk buffers come from one file-scope device array of fixed size
// instead of the tree's grown-on-demand buffers.  Every process that loads
// this library holds the array on every GPU it uses until it exits.
namespace trevr2 {

constexpr size_t kNoAllocScratchBytes = size_t(16) << 20;  // 16 MiB per device
constexpr int kNoAllocSources = 256;  // source records per warp and pass

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Device address of the array on the current device.  In host code the
// array's name is only a host-side stand-in, so its address is looked up,
// with the device current, on every call: a cached address would go stale
// if the device's context were reset and the module loaded again.  The
// first lookup on a device loads the library's module there.
static int noalloc_scratch(void** out) {
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(walk scratch)");
  *out = p;
  return TREVR2_OK;
}

static int launch_walk_noalloc(Tree* t, Table* tb, const int64_t* active, int64_t A, int nside,
                               float theta, const int* bsel, int nbsel, uint32_t flags, float* J,
                               cudaStream_t st) {
  void* scratch = nullptr;
  T2_CHECK(noalloc_scratch(&scratch));
  WalkArgs a;
  fill_walk_args(t, tb, nside, theta, bsel, nbsel, flags, kNoAllocSources, &a);
  a.active = active;
  a.A = A;
  a.J = J;
  const void* fn = walk_kernel(t->nbp, kWalkWarps, false);
  const size_t smem = walk_smem(kWalkWarps, a.stack_ints, a.npix, a.max_depth);
  int per_sm = 0, sms = 0;
  T2_CHECK(config_walk_kernel(fn, kWalkWarps, smem, &per_sm, &sms));
  // The grid is capped by what the fixed array holds; the kernel loops over
  // receivers and passes over sources, so any A and any source count fit.
  const size_t per_block = walk_buffer_bytes(kWalkWarps, a.M);
  const int64_t max_blocks = int64_t(kNoAllocScratchBytes / per_block);
  if (max_blocks < 1) {
    set_error("trevr2_J_noalloc: one block needs %zu bytes of walk buffers, the fixed array "
              "holds %zu", per_block, kNoAllocScratchBytes);
    return TREVR2_EUNSUPPORTED;
  }
  int64_t blocks = int64_t(sms) * per_sm;
  blocks = std::min<int64_t>(blocks, (A + kWalkWarps - 1) / kWalkWarps);
  blocks = std::min<int64_t>(blocks, max_blocks);
  blocks = std::max<int64_t>(blocks, 1);
  const size_t warps = size_t(blocks) * kWalkWarps;
  place_walk_buffers(static_cast<char*>(scratch), warps, a.M, &a.srcU, &a.srcV, &a.srcT, &a.pixU);
  T2_CUDA(cudaMemsetAsync(t->counter, 0, sizeof(unsigned long long), st));
  void* args[] = {&a};
  T2_CUDA(cudaLaunchKernel(fn, dim3(unsigned(blocks)), dim3(kWalkWarps * 32), args, smem, st));
  note_launch();
  return TREVR2_OK;
}

}  // namespace trevr2

extern "C" int trevr2_J_noalloc(trevr2_tree* tree, const int64_t* active, int64_t A, int nside,
                                float theta, const int* bands, int nbsel, uint32_t flags,
                                float* J, void* stream) {
  clear_error();
  if (!tree) {
    set_error("trevr2_J_noalloc: tree is NULL");
    return TREVR2_EINVAL;
  }
  Tree* t = reinterpret_cast<Tree*>(tree);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  t->last_stream = st;
  if (A < 0 || (A > 0 && (!active || !J))) {
    set_error("trevr2_J_noalloc: A < 0 or NULL active/J");
    return TREVR2_EINVAL;
  }
  if (!valid_nside(nside)) {
    set_error("trevr2_J_noalloc: nside %d is not a power of two in [1, %d]", nside,
              TREVR2_MAX_NSIDE);
    return nside > TREVR2_MAX_NSIDE ? TREVR2_EUNSUPPORTED : TREVR2_EINVAL;
  }
  if (!(theta > 0.0f) || !std::isfinite(theta)) {
    set_error("trevr2_J_noalloc: theta must be positive and finite");
    return TREVR2_EINVAL;
  }
  if (flags & ~(TREVR2_SOFT | TREVR2_THICK | TREVR2_LINEAR | TREVR2_ASYNC)) {
    set_error("trevr2_J_noalloc: unknown flag bits 0x%x", flags);
    return TREVR2_EINVAL;
  }
  int bsel[TREVR2_MAX_BANDS];
  if (bands) {
    if (nbsel < 1 || nbsel > t->nb) {
      set_error("trevr2_J_noalloc: nbsel = %d outside [1, %d]", nbsel, t->nb);
      return TREVR2_EINVAL;
    }
    for (int b = 0; b < nbsel; ++b) {
      if (bands[b] < 0 || bands[b] >= t->nb) {
        set_error("trevr2_J_noalloc: band index %d outside [0, %d)", bands[b], t->nb);
        return TREVR2_EINVAL;
      }
      bsel[b] = bands[b];
    }
  } else {
    nbsel = t->nb;
    for (int b = 0; b < nbsel; ++b) bsel[b] = b;
  }
  if (A == 0) return TREVR2_OK;
  Table* tb = nullptr;
  const bool linear = (flags & TREVR2_LINEAR) != 0;
  for (Table& cand : t->tables)
    if (cand.nside == nside && cand.linear == linear) tb = &cand;
  if (!tb) {
    set_error(linear ? "trevr2_J_noalloc: no linear-average tables for nside %d; make one "
                       "trevr2_J call with TREVR2_LINEAR and this nside first (this entry point "
                       "never allocates)"
                     : "trevr2_J_noalloc: no tables for nside %d; call trevr2_prepare(tree, %d) "
                       "first (this entry point never allocates)",
              nside, nside);
    return TREVR2_EINVAL;
  }
  T2_CHECK(launch_walk_noalloc(t, tb, active, A, nside, theta, bsel, nbsel, flags, J, st));
  if (flags & TREVR2_ASYNC) return TREVR2_OK;
  return read_status(t, st);
}
