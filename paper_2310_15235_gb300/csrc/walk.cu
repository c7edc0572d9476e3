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

#include "healpix.cuh"
#include "internal.cuh"

namespace trevr2 {

constexpr int kWalkWarps = 8;                 // warps per block
constexpr int kSrcCapacity = 1024;            // sources held per warp and pass
constexpr float kFourPi = 12.566370614359172f;

struct WalkArgs {
  const NodeW* nodes;
  const float4* csrc;
  const double* c64;
  const double* B64;
  const float* Lnode;
  const float* alpha_leaf;
  const float* alpha_tab;
  const float4* pos32;
  const double* pos64;
  const float* Lelem;
  const int* inv;
  const float* hn;
  const float* km;
  const float4* dirs;
  const int64_t* active;
  int64_t A;
  int64_t N;
  int nside, npix, P;
  float theta, theta2;
  double theta64;
  float guard_abs, guard_rel;
  uint32_t flags;
  int nb, nbsel;
  int bsel[TREVR2_MAX_BANDS];
  double inv_size2;
  double size;
  float* J;
  SrcEntry* srcU;
  int* pixU;
  SrcEntry* srcV;
  int M;
  int stack_ints;   // per warp
  int max_depth;
  uint32_t* status;
  unsigned long long* counter;
};

__device__ __forceinline__ float3 node_ext(uint32_t meta) {
  const int d = int(meta & kMetaDepthMask);
  return make_float3(__int_as_float((127 - splits_on_axis(d, 0)) << 23),
                     __int_as_float((127 - splits_on_axis(d, 1)) << 23),
                     __int_as_float((127 - splits_on_axis(d, 2)) << 23));
}

// FP64 opening decision, the definition evaluated without contraction.
__device__ __noinline__ bool opens64(const WalkArgs& a, int q, const NodeW& nd, int si) {
  const float3 e = node_ext(nd.meta);
  const double ext[3] = {double(e.x), double(e.y), double(e.z)};
  double s = 0.0;
  for (int k = 0; k < 3; ++k) {
    const double lo = double(nd.lo[k]), hi = __dadd_rn(lo, ext[k]);
    const double x = a.pos64[3 * int64_t(si) + k];
    double dd = 0.0;
    if (x < lo) dd = __dsub_rn(lo, x);
    else if (x > hi) dd = __dsub_rn(x, hi);
    s = __dadd_rn(s, __dmul_rn(dd, dd));
  }
  const double d = sqrt(s);
  return (d == 0.0) || (a.B64[q] > __dmul_rn(a.theta64, d));
}

// Coordinates for decisions on beams that lie in a plane of constant x[c]
// (a zero beam component): half-open boxes [lo, hi) hold the beam iff
// lo <= x[c] < hi, decided as on the FP64 position.  Box faces are
// multiples of 2^-21, exact in FP32, and rounding to nearest never carries a
// coordinate across one; the FP32 value only disagrees when it lands on a
// face that the FP64 value lies just below, and then the next float below
// restores the FP64 answer.
__device__ __forceinline__ float3 grazing_coords(const WalkArgs& a, int si, float3 x) {
  const double* p = a.pos64 + 3 * int64_t(si);
  float g[3] = {x.x, x.y, x.z};
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const double f = double(g[c]) * 2097152.0;
    if (f == floor(f) && p[c] < double(g[c])) g[c] = nextafterf(g[c], -INFINITY);
  }
  return make_float3(g[0], g[1], g[2]);
}

// Sec. 2.5.2: open iff d == 0 or B > theta d.
__device__ __forceinline__ bool cell_opens(const WalkArgs& a, int q, const NodeW& nd, float3 x,
                                           int si) {
  const float3 e = node_ext(nd.meta);
  const float dx = fmaxf(0.0f, fmaxf(nd.lo[0] - x.x, x.x - (nd.lo[0] + e.x)));
  const float dy = fmaxf(0.0f, fmaxf(nd.lo[1] - x.y, x.y - (nd.lo[1] + e.y)));
  const float dz = fmaxf(0.0f, fmaxf(nd.lo[2] - x.z, x.z - (nd.lo[2] + e.z)));
  const float d2 = dx * dx + dy * dy + dz * dz;
  if (d2 == 0.0f) return true;
  const float B = nd.B;
  const float margin = B * B - a.theta2 * d2;
  const float g = 2.2f * B * (a.guard_abs + a.guard_rel * B);
  if (fabsf(margin) > g) return margin > 0.0f;
  return opens64(a, q, nd, si);
}

// Eq. intint as a kernel of r for an element of size h (normalised units).
__device__ float soft_kernel(float r, float h) {
  const float x = r / (0.48860251190292f * h);
  float g;
  if (x == 1.0f) {
    g = 0.5f;
  } else if (x <= 2.0f) {
    const float xm = x - 1.0f, xp = x + 1.0f;
    g = 0.5f * (1.0f + (x * x - 1.0f) / (4.0f * x) * logf((xm * xm) / (xp * xp)));
  } else {
    // sum_{m>=1} x^{-2m}/(4m^2-1): the same function without the cancellation
    const float ix2 = 1.0f / (x * x);
    float xm = 1.0f, s = 0.0f;
    for (int m = 1; m < 64; ++m) {
      xm *= ix2;
      const float term = xm / float(4 * m * m - 1);
      s += term;
      if (term < 1e-9f * s) break;
    }
    g = s;
  }
  return g / (h * h);
}

// Bin one source: beam, projected distance, r/s, kernel.  Returns false for
// a source on top of the receiver (r == 0) or with s <= 0.
__device__ __forceinline__ bool make_source(const WalkArgs& a, float3 p, const double* p64,
                                            float3 x, int si, int ref, SrcEntry& out, int& pix) {
  const float vx = p.x - x.x, vy = p.y - x.y, vz = p.z - x.z;
  const float r2 = vx * vx + vy * vy + vz * vz;
  if (!(r2 > 0.0f)) return false;
  const float r = sqrtf(r2);
  int k = hp_vec2pix_f32(a.nside, vx, vy, vz, hp_guard(a.nside, r));
  if (k < 0) {
    const double* x64 = a.pos64 + 3 * int64_t(si);
    k = hp_vec2pix_f64(a.nside, __dsub_rn(p64[0], x64[0]), __dsub_rn(p64[1], x64[1]),
                       __dsub_rn(p64[2], x64[2]));
  }
  const float4 n = a.dirs[k];
  const float s = vx * n.x + vy * n.y + vz * n.z;
  if (!(s > 0.0f)) return false;
  out.s = s;
  out.rs = r / s;
  out.w = (a.flags & TREVR2_SOFT) ? soft_kernel(r, a.hn[si]) : 1.0f / (kFourPi * r2);
  out.ref = ref;
  pix = k;
  return true;
}

__device__ __forceinline__ int warp_incl_scan(int v, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int u = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += u;
  }
  return v;
}

// Phase S for the sources whose running index is in [lo, lo + M).  Returns
// the total number of sources of this receiver (warp-uniform).
__device__ int phase_sources(const WalkArgs& a, float3 x, int si, int lane, int* stk, int cap,
                             SrcEntry* U, int* Up, int lo) {
  int sp = 1;
  if (lane == 0) stk[0] = 0;
  __syncwarp();
  int emitted = 0;
  const unsigned lt = (1u << lane) - 1u;
  while (sp > 0) {
    const int k = min(32, sp);
    const int q = lane < k ? stk[sp - 1 - lane] : -1;
    sp -= k;
    __syncwarp();
    int npush = 0, child = -1, leaf_first = 0, leaf_count = 0;
    bool emit_node = false;
    SrcEntry ent;
    int pix = 0;
    if (q >= 0) {
      const NodeW nd = a.nodes[q];
      if (nd.meta & kMetaHasL) {
        if (!cell_opens(a, q, nd, x, si)) {
          const float4 c = a.csrc[q];
          emit_node = make_source(a, make_float3(c.x, c.y, c.z), a.c64 + 3 * int64_t(q), x, si, q,
                                  ent, pix);
        } else if (nd.meta & kMetaLeaf) {
          leaf_first = nd.aux;
          leaf_count = nd.count;
        } else {
          npush = 2;
          child = nd.child;
        }
      }
    }
    // push opened halves
    const int incl = warp_incl_scan(npush, lane);
    const int tot = __shfl_sync(0xffffffffu, incl, 31);
    if (npush) {
      const int pos = sp + incl - npush;
      if (pos + 2 <= cap) {
        stk[pos] = child + 1;
        stk[pos + 1] = child;
      } else {
        atomicOr(a.status, kStatusStackOverflow);
      }
    }
    sp = min(sp + tot, cap);
    // accepted luminous cells
    {
      const unsigned m = __ballot_sync(0xffffffffu, emit_node);
      const int idx = emitted + __popc(m & lt) - lo;
      if (emit_node && idx >= 0 && idx < a.M) {
        U[idx] = ent;
        Up[idx] = pix;
      }
      emitted += __popc(m);
    }
    // luminous elements of opened leaves
    int maxc = leaf_count;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) maxc = max(maxc, __shfl_xor_sync(0xffffffffu, maxc, o));
    for (int e = 0; e < maxc; ++e) {
      bool em = false;
      if (e < leaf_count) {
        const int sj = leaf_first + e;
        const float4 pj = a.pos32[sj];
        if (pj.w > 0.0f && sj != si)
          em = make_source(a, make_float3(pj.x, pj.y, pj.z), a.pos64 + 3 * int64_t(sj), x, si,
                           sj | kRefElement, ent, pix);
      }
      const unsigned m = __ballot_sync(0xffffffffu, em);
      const int idx = emitted + __popc(m & lt) - lo;
      if (em && idx >= 0 && idx < a.M) {
        U[idx] = ent;
        Up[idx] = pix;
      }
      emitted += __popc(m);
    }
    __syncwarp();
  }
  return emitted;
}

// Bucket the n sources of U by beam into V; off[k] ends as the end of
// bucket k (its start is off[k-1], or 0).  Each bucket is sorted by s.
__device__ void bin_sources(const WalkArgs& a, int lane, const SrcEntry* U, const int* Up, int n,
                            SrcEntry* V, int* off) {
  const int npix = a.npix;
  for (int k = lane; k < npix; k += 32) off[k] = 0;
  __syncwarp();
  for (int e = lane; e < n; e += 32) atomicAdd(&off[Up[e]], 1);
  __syncwarp();
  // exclusive scan of the bucket sizes
  const int per = (npix + 31) / 32;
  const int b0 = min(lane * per, npix), b1 = min(b0 + per, npix);
  int sum = 0;
  for (int k = b0; k < b1; ++k) sum += off[k];
  const int incl = warp_incl_scan(sum, lane);
  int run = incl - sum;
  for (int k = b0; k < b1; ++k) {
    const int c = off[k];
    off[k] = run;
    run += c;
  }
  __syncwarp();
  for (int e = lane; e < n; e += 32) {
    const int slot = atomicAdd(&off[Up[e]], 1);
    V[slot] = U[e];
  }
  __syncwarp();
  // insertion sort of each bucket by projected distance
  for (int k = lane; k < npix; k += 32) {
    const int s0 = k ? off[k - 1] : 0, s1 = off[k];
    for (int i = s0 + 1; i < s1; ++i) {
      const SrcEntry v = V[i];
      int j = i - 1;
      while (j >= s0 && V[j].s > v.s) {
        V[j + 1] = V[j];
        --j;
      }
      V[j + 1] = v;
    }
  }
  __syncwarp();
}

template <int NBP>
struct BandVec {
  float v[NBP];
};

template <int NBP>
__device__ __forceinline__ BandVec<NBP> load_bands(const float* p) {
  BandVec<NBP> r;
  if constexpr (NBP == 4) {
    const float4 t = *reinterpret_cast<const float4*>(p);
    r.v[0] = t.x; r.v[1] = t.y; r.v[2] = t.z; r.v[3] = t.w;
  } else if constexpr (NBP == 2) {
    const float2 t = *reinterpret_cast<const float2*>(p);
    r.v[0] = t.x; r.v[1] = t.y;
  } else {
    r.v[0] = *p;
  }
  return r;
}

// Phase A: lanes take beams (those with sources) from a per-warp counter.
template <int NBP>
__device__ void phase_absorb(const WalkArgs& a, float3 x, int si, int lane, int* lstk,
                             const SrcEntry* V, const int* off, int* next_beam, float* Js,
                             float* Jc) {
  int k = lane;
  for (;;) {
    while (k < a.npix && (k ? off[k - 1] : 0) == off[k]) k = atomicAdd(next_beam, 1);
    if (k >= a.npix) break;
    int ptr = k ? off[k - 1] : 0;
    const int end = off[k];
    const float smax = V[end - 1].s;
    const float4 dn = a.dirs[k];
    const int pair = __float_as_int(dn.w);
    const float n[3] = {dn.x, dn.y, dn.z};
    float inv[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) inv[c] = n[c] != 0.0f ? 1.0f / n[c] : 0.0f;
    const float xv[3] = {x.x, x.y, x.z};
    float tau[NBP];
#pragma unroll
    for (int b = 0; b < NBP; ++b) tau[b] = 0.0f;
    int sp = 1;
    lstk[0] = 0;
    while (sp > 0 && ptr < end) {
      const int q = lstk[--sp];
      const NodeW nd = a.nodes[q];
      if (!(nd.meta & kMetaHasAlpha)) continue;
      const float3 e = node_ext(nd.meta);
      const float ext[3] = {e.x, e.y, e.z};
      float t0 = 0.0f, t1 = smax;
      bool hit = true;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const float lo = nd.lo[c], hi = lo + ext[c];
        if (n[c] == 0.0f) {
          hit &= (lo <= xv[c]) && (xv[c] < hi);  // half-open box for a grazing beam
        } else {
          const float ta = (lo - xv[c]) * inv[c], tb = (hi - xv[c]) * inv[c];
          t0 = fmaxf(t0, fminf(ta, tb));
          t1 = fminf(t1, fmaxf(ta, tb));
        }
      }
      if (!hit || !(t0 < t1)) continue;
      if (!(nd.meta & kMetaLeaf) && cell_opens(a, q, nd, x, si)) {
        // near half (the side of the receiver) on top of the stack
        const int axis = int(nd.meta & kMetaDepthMask) % 3;
        const float mid = nd.lo[axis] + 0.5f * ext[axis];
        const bool lower_first = xv[axis] < mid;
        lstk[sp] = lower_first ? nd.child + 1 : nd.child;
        lstk[sp + 1] = lower_first ? nd.child : nd.child + 1;
        sp += 2;
        continue;
      }
      const BandVec<NBP> al = (nd.meta & kMetaLeaf)
                                  ? load_bands<NBP>(a.alpha_leaf + int64_t(q) * NBP)
                                  : load_bands<NBP>(a.alpha_tab + (int64_t(nd.aux) * a.P + pair) * NBP);
      while (ptr < end) {
        const SrcEntry src = V[ptr];
        if (!(src.s < t1)) break;
        const float ds = fmaxf(0.0f, src.s - t0);
        const float* Lp = (src.ref & kRefElement) ? a.Lelem + int64_t(src.ref & 0x7fffffff) * NBP
                                                  : a.Lnode + int64_t(src.ref) * NBP;
        const BandVec<NBP> L = load_bands<NBP>(Lp);
#pragma unroll
        for (int b = 0; b < NBP; ++b) {
          const float term = L.v[b] * src.w * expf(-(tau[b] + al.v[b] * ds) * src.rs);
          const float y = term - Jc[b];
          const float t = Js[b] + y;
          Jc[b] = (t - Js[b]) - y;
          Js[b] = t;
        }
        ++ptr;
      }
#pragma unroll
      for (int b = 0; b < NBP; ++b) tau[b] += al.v[b] * (t1 - t0);
    }
    // sources beyond the last absorbing cell of the beam
    while (ptr < end) {
      const SrcEntry src = V[ptr];
      const float* Lp = (src.ref & kRefElement) ? a.Lelem + int64_t(src.ref & 0x7fffffff) * NBP
                                                : a.Lnode + int64_t(src.ref) * NBP;
      const BandVec<NBP> L = load_bands<NBP>(Lp);
#pragma unroll
      for (int b = 0; b < NBP; ++b) {
        const float term = L.v[b] * src.w * expf(-tau[b] * src.rs);
        const float y = term - Jc[b];
        const float t = Js[b] + y;
        Jc[b] = (t - Js[b]) - y;
        Js[b] = t;
      }
      ++ptr;
    }
    k = atomicAdd(next_beam, 1);
  }
}

template <int NBP>
__global__ void __launch_bounds__(kWalkWarps * 32) k_walk(WalkArgs a) {
  extern __shared__ int smem[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t gw = int64_t(blockIdx.x) * kWalkWarps + wib;
  int* wsm = smem + wib * (a.stack_ints + a.npix + 1);
  int* stk = wsm;
  int* off = wsm + a.stack_ints;
  int* next_beam = off + a.npix;
  int* lstk = stk + lane * (a.max_depth + 2);
  SrcEntry* U = a.srcU + gw * a.M;
  int* Up = a.pixU + gw * a.M;
  SrcEntry* V = a.srcV + gw * a.M;
  for (;;) {
    unsigned long long slot = 0;
    if (lane == 0) slot = atomicAdd(a.counter, 1ull);
    slot = __shfl_sync(0xffffffffu, slot, 0);
    if (slot >= (unsigned long long)a.A) break;
    const int64_t io = a.active[slot];
    if (io < 0 || io >= a.N) {
      if (lane == 0) atomicOr(a.status, kStatusBadActive);
      if (lane < a.nbsel) a.J[int64_t(slot) * a.nbsel + lane] = __int_as_float(0x7fc00000);
      continue;
    }
    const int si = a.inv[io];
    const float4 xr = a.pos32[si];
    // the receiver in FP32, on the FP64 side of every box face
    const float3 x = grazing_coords(a, si, make_float3(xr.x, xr.y, xr.z));
    float Js[NBP], Jc[NBP];
#pragma unroll
    for (int b = 0; b < NBP; ++b) Js[b] = Jc[b] = 0.0f;
    for (int lo = 0;; lo += a.M) {
      const int total = phase_sources(a, x, si, lane, stk, a.stack_ints, U, Up, lo);
      const int n = min(total - lo, a.M);
      if (n > 0) {
        bin_sources(a, lane, U, Up, n, V, off);
        if (lane == 0) *next_beam = 32;
        __syncwarp();
        phase_absorb<NBP>(a, x, si, lane, lstk, V, off, next_beam, Js, Jc);
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
      a.J[int64_t(slot) * a.nbsel + lane] = float(v);
    }
  }
}

static bool valid_nside(int nside) {
  return nside >= 1 && nside <= TREVR2_MAX_NSIDE && (nside & (nside - 1)) == 0;
}

static int launch_walk(Tree* t, Table* tb, const int64_t* active, int64_t A, int nside,
                       float theta, const int* bsel, int nbsel, uint32_t flags, float* J,
                       cudaStream_t st) {
  int dev = 0, sms = 0;
  T2_CUDA(cudaGetDevice(&dev));
  T2_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  WalkArgs a;
  a.nodes = t->nodes;
  a.csrc = t->csrc;
  a.c64 = t->c64;
  a.B64 = t->B64;
  a.Lnode = t->Lnode;
  a.alpha_leaf = t->alpha_leaf;
  a.alpha_tab = tb->alpha;
  a.pos32 = t->pos32;
  a.pos64 = t->pos64;
  a.Lelem = t->Lelem;
  a.inv = t->inv;
  a.hn = t->hn;
  a.km = t->km;
  a.dirs = tb->dirs;
  a.active = active;
  a.A = A;
  a.N = t->N;
  a.nside = nside;
  a.npix = 12 * nside * nside;
  a.P = a.npix / 2;
  a.theta = theta;
  a.theta2 = theta * theta;
  a.theta64 = double(theta);
  a.guard_abs = 2e-7f * theta + 2e-7f;
  a.guard_rel = 2e-6f;
  a.flags = flags;
  a.nb = t->nb;
  a.nbsel = nbsel;
  for (int b = 0; b < TREVR2_MAX_BANDS; ++b) a.bsel[b] = b < nbsel ? bsel[b] : 0;
  a.inv_size2 = 1.0 / (t->size * t->size);
  a.size = t->size;
  a.J = J;
  a.M = kSrcCapacity;
  a.max_depth = t->max_depth;
  a.stack_ints = 64 * (t->max_depth + 2);
  a.status = t->status;
  a.counter = t->counter;
  const size_t smem = size_t(kWalkWarps) * (a.stack_ints + a.npix + 1) * sizeof(int);
  int max_smem = 0;
  T2_CUDA(cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  if (smem > size_t(max_smem)) {
    set_error("trevr2_J: tree depth %d with nside %d needs %zu bytes of shared memory per block",
              t->max_depth, nside, smem);
    return TREVR2_EUNSUPPORTED;
  }
  const void* fn = t->nbp == 1 ? reinterpret_cast<const void*>(&k_walk<1>)
                 : t->nbp == 2 ? reinterpret_cast<const void*>(&k_walk<2>)
                               : reinterpret_cast<const void*>(&k_walk<4>);
  T2_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
  int per_sm = 0;
  T2_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kWalkWarps * 32, smem));
  if (per_sm < 1) per_sm = 1;
  int64_t blocks = int64_t(sms) * per_sm;
  blocks = std::min<int64_t>(blocks, (A + kWalkWarps - 1) / kWalkWarps);
  blocks = std::max<int64_t>(blocks, 1);
  const size_t warps = size_t(blocks) * kWalkWarps;
  const size_t need = warps * a.M * (2 * sizeof(SrcEntry) + sizeof(int));
  if (t->scratch_bytes < need) {
    if (t->scratch) cudaFreeAsync(t->scratch, st);
    t->scratch = nullptr;
    t->scratch_bytes = 0;
    cudaError_t e = cudaMallocAsync(&t->scratch, need, st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync(walk buffers)");
    t->scratch_bytes = need;
  }
  char* base = static_cast<char*>(t->scratch);
  a.srcU = reinterpret_cast<SrcEntry*>(base);
  a.srcV = reinterpret_cast<SrcEntry*>(base + warps * a.M * sizeof(SrcEntry));
  a.pixU = reinterpret_cast<int*>(base + 2 * warps * a.M * sizeof(SrcEntry));
  T2_CUDA(cudaMemsetAsync(t->counter, 0, sizeof(unsigned long long), st));
  void* args[] = {&a};
  T2_CUDA(cudaLaunchKernel(fn, dim3(unsigned(blocks)), dim3(kWalkWarps * 32), args, smem, st));
  note_launch();
  return TREVR2_OK;
}

static int read_status(Tree* t, cudaStream_t st) {
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
  set_error("trevr2: device status 0x%x", s);
  return TREVR2_EINTERNAL;
}

}  // namespace trevr2

using namespace trevr2;

extern "C" int trevr2_J(trevr2_tree* tree, const int64_t* active, int64_t A, int nside, float theta,
                        const int* bands, int nbsel, uint32_t flags, float* J, void* stream) {
  clear_error();
  if (!tree) {
    set_error("trevr2_J: tree is NULL");
    return TREVR2_EINVAL;
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
  if (flags & ~(TREVR2_SOFT | TREVR2_THICK | TREVR2_ASYNC)) {
    set_error("trevr2_J: unknown flag bits 0x%x", flags);
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
  T2_CHECK(ensure_table(t, nside, st, &tb));
  T2_CHECK(launch_walk(t, tb, active, A, nside, theta, bsel, nbsel, flags, J, st));
  if (flags & TREVR2_ASYNC) return TREVR2_OK;
  return read_status(t, st);
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
#include <mutex>

namespace trevr2 {

constexpr size_t kNoAllocScratchBytes = size_t(16) << 20;  // 16 MiB per device
constexpr int kNoAllocSources = 256;  // source records per warp and pass
constexpr int kNoAllocMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

static std::mutex g_noalloc_mu;
static void* g_noalloc_ptr[kNoAllocMaxDevices] = {};

// Device address of the array for the current device.  In host code the
// array's name is only a host-side stand-in, so the address is looked up
// once per device (with that device current) and cached.
static int noalloc_scratch(void** out) {
  int dev = 0;
  T2_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kNoAllocMaxDevices) {
    set_error("trevr2_J_noalloc: device ordinal %d above %d", dev, kNoAllocMaxDevices - 1);
    return TREVR2_EUNSUPPORTED;
  }
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(walk scratch)");
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return TREVR2_OK;
}

static int launch_walk_noalloc(Tree* t, Table* tb, const int64_t* active, int64_t A, int nside,
                               float theta, const int* bsel, int nbsel, uint32_t flags, float* J,
                               cudaStream_t st) {
  void* scratch = nullptr;
  T2_CHECK(noalloc_scratch(&scratch));
  int dev = 0, sms = 0;
  T2_CUDA(cudaGetDevice(&dev));
  T2_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  WalkArgs a;
  a.nodes = t->nodes;
  a.csrc = t->csrc;
  a.c64 = t->c64;
  a.B64 = t->B64;
  a.Lnode = t->Lnode;
  a.alpha_leaf = t->alpha_leaf;
  a.alpha_tab = tb->alpha;
  a.pos32 = t->pos32;
  a.pos64 = t->pos64;
  a.Lelem = t->Lelem;
  a.inv = t->inv;
  a.hn = t->hn;
  a.km = t->km;
  a.dirs = tb->dirs;
  a.active = active;
  a.A = A;
  a.N = t->N;
  a.nside = nside;
  a.npix = 12 * nside * nside;
  a.P = a.npix / 2;
  a.theta = theta;
  a.theta2 = theta * theta;
  a.theta64 = double(theta);
  a.guard_abs = 2e-7f * theta + 2e-7f;
  a.guard_rel = 2e-6f;
  a.flags = flags;
  a.nb = t->nb;
  a.nbsel = nbsel;
  for (int b = 0; b < TREVR2_MAX_BANDS; ++b) a.bsel[b] = b < nbsel ? bsel[b] : 0;
  a.inv_size2 = 1.0 / (t->size * t->size);
  a.size = t->size;
  a.J = J;
  a.M = kNoAllocSources;
  a.max_depth = t->max_depth;
  a.stack_ints = 64 * (t->max_depth + 2);
  a.status = t->status;
  a.counter = t->counter;
  const size_t smem = size_t(kWalkWarps) * (a.stack_ints + a.npix + 1) * sizeof(int);
  int max_smem = 0;
  T2_CUDA(cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  if (smem > size_t(max_smem)) {
    set_error("trevr2_J_noalloc: tree depth %d with nside %d needs %zu bytes of shared memory",
              t->max_depth, nside, smem);
    return TREVR2_EUNSUPPORTED;
  }
  const void* fn = t->nbp == 1 ? reinterpret_cast<const void*>(&k_walk<1>)
                 : t->nbp == 2 ? reinterpret_cast<const void*>(&k_walk<2>)
                               : reinterpret_cast<const void*>(&k_walk<4>);
  T2_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
  int per_sm = 0;
  T2_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kWalkWarps * 32, smem));
  if (per_sm < 1) per_sm = 1;
  // The grid is capped by what the fixed array holds; the kernel loops over
  // receivers and passes over sources, so any A and any source count fit.
  const size_t per_block = size_t(kWalkWarps) * a.M * (2 * sizeof(SrcEntry) + sizeof(int));
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
  char* base = static_cast<char*>(scratch);
  a.srcU = reinterpret_cast<SrcEntry*>(base);
  a.srcV = reinterpret_cast<SrcEntry*>(base + warps * a.M * sizeof(SrcEntry));
  a.pixU = reinterpret_cast<int*>(base + 2 * warps * a.M * sizeof(SrcEntry));
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
  if (flags & ~(TREVR2_SOFT | TREVR2_THICK | TREVR2_ASYNC)) {
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
  for (Table& cand : t->tables)
    if (cand.nside == nside) tb = &cand;
  if (!tb) {
    set_error("trevr2_J_noalloc: no tables for nside %d; call trevr2_prepare(tree, %d) first "
              "(this entry point never allocates)", nside, nside);
    return TREVR2_EINVAL;
  }
  T2_CHECK(launch_walk_noalloc(t, tb, active, A, nside, theta, bsel, nbsel, flags, J, st));
  if (flags & TREVR2_ASYNC) return TREVR2_OK;
  return read_status(t, st);
}
