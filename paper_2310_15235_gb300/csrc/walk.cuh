// Device pieces of the TREVR2 walk shared by the forward walk (walk.cu) and
// the adjoint walk (adjoint.cu): walk arguments, the opening criterion
// (Sec. 2.5.2), the source kernel (Eq. intint), source binning by HEALPix
// beam (Sec. 2.5.1) and the warp-cooperative source phase.
#pragma once

#include <cfloat>
#include <cmath>

#include "healpix.cuh"
#include "internal.cuh"

namespace trevr2 {

constexpr int kWalkWarps = 4;                 // warps per block
// Resident warps per SM the walk kernels are compiled for: 7 blocks of 4
// warps (72 registers a thread) measured faster than 6 at 80 registers and
// than 8 at 64 registers, which spills.
constexpr int kWalkWarpsPerSM = 28;
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
  const int* order;  // walk order of the receivers (NULL: as given)
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
  float* srcT;      // [warps][M][4] optical depth tau_k(s) of every staged source
  double* origin64; // [warps][kOriginWords] per-bucket walk: FP64 centre, r_pp,
                    // directed beam (unit vector, pixel or -1)
  int M;
  int stack_ints;   // per warp
  int src_stack_cap;  // entries of the source cut's stack used (<= stack_ints)
  int max_depth;
  uint32_t* status;
  unsigned long long* counter;
  // complex source model (per-bucket walk with TREVR2_CSM; NULL when off)
  const float* csm_tau;  // [n][npix][nbp]
  const float* csm_d;    // [n][npix]
  const int* csm_anti;   // [npix]
};

__device__ __forceinline__ float3 node_ext(uint32_t meta) {
  const int d = int(meta & kMetaDepthMask);
  const int q = (d * 21846) >> 16;  // d / 3 for d < 64
  const int r = int((meta >> kMetaAxisShift) & 3u);  // d % 3
  const float e = __int_as_float((127 - q) << 23);
  return make_float3(r > 0 ? 0.5f * e : e, r > 1 ? 0.5f * e : e, e);
}

// Chord [t0, t1) of the beam x + t n (inv = 1/n, 0 where n = 0) with the box
// of nd, clipped to [0, tmax]; half-open boxes decide grazing beams.
__device__ __forceinline__ bool beam_chord(const NodeW& nd, const float xv[3], const float n[3],
                                           const float inv[3], float tmax, float& t0,
                                           float& t1) {
  const float3 e = node_ext(nd.meta);
  const float ext[3] = {e.x, e.y, e.z};
  t0 = 0.0f;
  t1 = tmax;
  bool hit = true;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const float lo = nd.lo[c], hi = lo + ext[c];
    if (n[c] == 0.0f) {
      hit &= (lo <= xv[c]) && (xv[c] < hi);
    } else {
      const float ta = (lo - xv[c]) * inv[c], tb = (hi - xv[c]) * inv[c];
      t0 = fmaxf(t0, fminf(ta, tb));
      t1 = fminf(t1, fmaxf(ta, tb));
    }
  }
  return hit && (t0 < t1);
}

// The halves of an opened node that a beam (x + t n, t in [t0, t1), the
// node's own chord) crosses and that hold some absorption, which half the
// beam meets first (the receiver's side), and each half's chord [lt0, lt1),
// [ut0, ut1).  The crossing time of the split plane is the face time each
// half computes for itself and min/max are exact, so these are bit for bit
// the chords the halves' own slab tests give.
__device__ __forceinline__ void crossed_halves(const NodeW& nd, const float xv[3], const float n[3],
                                               const float inv[3], float t0, float t1,
                                               bool& lower_first, bool& lower_hit,
                                               bool& upper_hit, float& lt0, float& lt1,
                                               float& ut0, float& ut1) {
  const int axis = int(nd.meta & kMetaDepthMask) % 3;
  const float3 e = node_ext(nd.meta);
  const float lo = axis == 0 ? nd.lo[0] : (axis == 1 ? nd.lo[1] : nd.lo[2]);
  const float ex = axis == 0 ? e.x : (axis == 1 ? e.y : e.z);
  const float xa = axis == 0 ? xv[0] : (axis == 1 ? xv[1] : xv[2]);
  const float na = axis == 0 ? n[0] : (axis == 1 ? n[1] : n[2]);
  const float ia = axis == 0 ? inv[0] : (axis == 1 ? inv[1] : inv[2]);
  const float mid = lo + 0.5f * ex;
  lower_first = xa < mid;
  lt0 = ut0 = t0;
  lt1 = ut1 = t1;
  if (na == 0.0f) {
    lower_hit = lower_first;
    upper_hit = !lower_first;
  } else {
    const float tm = (mid - xa) * ia;
    const float a1 = fminf(t1, tm), b0 = fmaxf(t0, tm);  // [t0, a1) before, [b0, t1) after
    if (na > 0.0f) {
      lt1 = a1;
      ut0 = b0;
    } else {
      ut1 = a1;
      lt0 = b0;
    }
    lower_hit = lt0 < lt1;
    upper_hit = ut0 < ut1;
  }
  lower_hit &= (nd.meta & kMetaChild0Alpha) != 0;
  upper_hit &= (nd.meta & kMetaChild1Alpha) != 0;
}


// Phase A forms: nx = x * inv per beam, slab times by one FMA per face.
__device__ __forceinline__ bool beam_chord_fx(const NodeW& nd, const float xv[3], const float n[3],
                                              const float inv[3], const float nx[3], float tmax,
                                              float& t0, float& t1) {
  const float3 e = node_ext(nd.meta);
  const float ext[3] = {e.x, e.y, e.z};
  t0 = 0.0f;
  t1 = tmax;
  bool hit = true;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const float lo = nd.lo[c], hi = lo + ext[c];
    if (n[c] == 0.0f) {
      hit &= (lo <= xv[c]) && (xv[c] < hi);
    } else {
      const float ta = fmaf(lo, inv[c], -nx[c]), tb = fmaf(hi, inv[c], -nx[c]);
      t0 = fmaxf(t0, fminf(ta, tb));
      t1 = fminf(t1, fmaxf(ta, tb));
    }
  }
  return hit && (t0 < t1);
}

// ex is the node's extent along its split axis (node_ext(meta).z: the split
// axis is the one bisected least often so far).  nx may be -inf on an axis
// with n = 0; it is only read on the others.  kBranchFree takes a grazing
// beam (n = 0 on the split axis) through the same arithmetic as the others
// (same decisions; faster, except in the p-p walk, which spills at its
// register limit and keeps the branch).
template <bool kBranchFree = true>
__device__ __forceinline__ void crossed_halves_fx(const NodeW& nd, const float xv[3], const float n[3],
                                                  const float inv[3], const float nx[3], float ex,
                                                  float t0, float t1, bool& lower_first,
                                                  bool& lower_hit, bool& upper_hit, float& lt0,
                                                  float& lt1, float& ut0, float& ut1) {
  const int axis = int((nd.meta >> kMetaAxisShift) & 3u);
  const float lo = axis == 0 ? nd.lo[0] : (axis == 1 ? nd.lo[1] : nd.lo[2]);
  const float xa = axis == 0 ? xv[0] : (axis == 1 ? xv[1] : xv[2]);
  const float na = axis == 0 ? n[0] : (axis == 1 ? n[1] : n[2]);
  const float ia = axis == 0 ? inv[0] : (axis == 1 ? inv[1] : inv[2]);
  const float nxa = axis == 0 ? nx[0] : (axis == 1 ? nx[1] : nx[2]);
  const float mid = lo + 0.5f * ex;
  lower_first = xa < mid;
  lt0 = ut0 = t0;
  lt1 = ut1 = t1;
  if (!kBranchFree && na == 0.0f) {
    lower_hit = lower_first;
    upper_hit = !lower_first;
  } else {
    // a grazing beam (na = 0) never reaches the split plane: +inf on the
    // receiver's side, -inf on the other, taken as a beam in +axis
    const float tm = na != 0.0f ? fmaf(mid, ia, -nxa) : (lower_first ? INFINITY : -INFINITY);
    const float a1 = fminf(t1, tm), b0 = fmaxf(t0, tm);
    if (na >= 0.0f) {
      lt1 = a1;
      ut0 = b0;
    } else {
      ut1 = a1;
      lt0 = b0;
    }
    lower_hit = lt0 < lt1;
    upper_hit = ut0 < ut1;
  }
  lower_hit &= (nd.meta & kMetaChild0Alpha) != 0;
  upper_hit &= (nd.meta & kMetaChild1Alpha) != 0;
}

// The receiver's ancestors, root first, into chain[] (shared memory, written
// by lane 0) by the same half-open decisions as the beams' near halves;
// returns the receiver's leaf.
__device__ __forceinline__ int build_chain(const NodeW* __restrict__ nodes, float3 x, int lane,
                                           NodeW* chain) {
  const float xv[3] = {x.x, x.y, x.z};
  const float zero3[3] = {0.0f, 0.0f, 0.0f};
  int leaf = 0;
  for (int d = 0;; ++d) {
    const NodeW nd = nodes[leaf];
    if (lane == 0) chain[d] = nd;
    if (nd.meta & kMetaLeaf) break;
    bool lower_first, lh, uh;
    float l0, l1, u0, u1;
    crossed_halves(nd, xv, zero3, zero3, 0.0f, 1.0f, lower_first, lh, uh, l0, l1, u0, u1);
    leaf = lower_first ? nd.child : nd.child + 1;
  }
  __syncwarp();
  return leaf;
}

// FP64 opening decision, the definition evaluated without contraction.
static __device__ __noinline__ bool opens64(const double* __restrict__ x64, double B,
                                            double theta, float lx, float ly, float lz,
                                            uint32_t meta) {
  const float3 e = node_ext(meta);
  const double ext[3] = {double(e.x), double(e.y), double(e.z)};
  const double lo3[3] = {double(lx), double(ly), double(lz)};
  double s = 0.0;
  for (int k = 0; k < 3; ++k) {
    const double lo = lo3[k], hi = __dadd_rn(lo, ext[k]);
    const double x = x64[k];
    double dd = 0.0;
    if (x < lo) dd = __dsub_rn(lo, x);
    else if (x > hi) dd = __dsub_rn(x, hi);
    s = __dadd_rn(s, __dmul_rn(dd, dd));
  }
  const double d = sqrt(s);
  return (d == 0.0) || (B > __dmul_rn(theta, d));
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

// The per-bucket walk's slot of warp w: [0..2] FP64 bucket centre, [3] FP64
// p-p radius, [4..6] unit vector of the directed beam, [7] its pixel (-1:
// none).
constexpr int kOriginWords = 8;

// The FP64 origin of a walk: the receiver's FP64 position, or (kBucket) the
// bucket centre in the slot of warp w = -1 - si.
template <bool kBucket>
__device__ __forceinline__ const double* origin64(const WalkArgs& a, int si) {
  if constexpr (kBucket) return a.origin64 + kOriginWords * int64_t(-1 - si);
  return a.pos64 + 3 * int64_t(si);
}

// FP64 distance from the FP64 origin x64 to a box, the definition without
// contraction, below r?
static __device__ __noinline__ bool box_within64(const double* __restrict__ x64, double r,
                                                 float lx, float ly, float lz, uint32_t meta) {
  const float3 e = node_ext(meta);
  const double ext[3] = {double(e.x), double(e.y), double(e.z)};
  const double lo3[3] = {double(lx), double(ly), double(lz)};
  double s = 0.0;
  for (int k = 0; k < 3; ++k) {
    const double lo = lo3[k], hi = __dadd_rn(lo, ext[k]);
    double dd = 0.0;
    if (x64[k] < lo) dd = __dsub_rn(lo, x64[k]);
    else if (x64[k] > hi) dd = __dsub_rn(x64[k], hi);
    s = __dadd_rn(s, __dmul_rn(dd, dd));
  }
  return sqrt(s) < r;
}

// Sec. 2.5.2: open iff d == 0 or B > theta d, seen from x (receiver si, or
// with kBucket the centre of the bucket that warp -1 - si walks).  With
// kPP and rpp > 0 (Sec. 2.4) a cell within the bucket's p-p radius opens
// too; the FP64 radius is the fourth word of the warp's origin slot.  e is
// the node's box extent.  d = 0 needs no test of its own: the margin is then
// B^2 > 0, and inside the guard band the FP64 decision opens at d = 0.
template <bool kBucket = false, bool kPP = false>
__device__ __forceinline__ bool cell_opens_e(const WalkArgs& a, int q, const NodeW& nd, float3 e,
                                             float3 x, int si, float rpp = 0.0f) {
  const float dx = fmaxf(0.0f, fmaxf(nd.lo[0] - x.x, x.x - (nd.lo[0] + e.x)));
  const float dy = fmaxf(0.0f, fmaxf(nd.lo[1] - x.y, x.y - (nd.lo[1] + e.y)));
  const float dz = fmaxf(0.0f, fmaxf(nd.lo[2] - x.z, x.z - (nd.lo[2] + e.z)));
  const float d2 = dx * dx + dy * dy + dz * dz;
  if constexpr (kBucket && kPP) {
    if (rpp > 0.0f) {
      const float m = d2 - rpp * rpp;
      if (fabsf(m) <= 1e-5f * rpp * rpp) {
        const double* o = origin64<true>(a, si);
        if (box_within64(o, o[3], nd.lo[0], nd.lo[1], nd.lo[2], nd.meta)) return true;
      } else if (m < 0.0f) {
        return true;
      }
    }
  }
  const float B = nd.B;
  const float margin = B * B - a.theta2 * d2;
  const float g = 2.2f * B * (a.guard_abs + a.guard_rel * B);
  if (fabsf(margin) > g) return margin > 0.0f;
  return opens64(origin64<kBucket>(a, si), a.B64[q], a.theta64, nd.lo[0], nd.lo[1], nd.lo[2], nd.meta);
}

template <bool kBucket = false, bool kPP = false>
__device__ __forceinline__ bool cell_opens(const WalkArgs& a, int q, const NodeW& nd, float3 x,
                                           int si, float rpp = 0.0f) {
  return cell_opens_e<kBucket, kPP>(a, q, nd, node_ext(nd.meta), x, si, rpp);
}

// Eq. intint as a kernel of r for an element of size h (normalised units).
static __device__ float soft_kernel(float r, float h) {
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
// a source on top of the receiver (r == 0) or with s <= 0.  From a bucket
// centre (kBucket) there is no kernel and r/s is the centre's, unused: w
// holds the projected distance s, each receiver of the bucket applies its
// own distance, and with kCSM the absorption key s moves to the cell's
// projected edge.
template <bool kBucket = false, bool kCSM = false>
__device__ __forceinline__ bool make_source(const WalkArgs& a, float3 p, const double* p64,
                                            float3 x, int si, int ref, SrcEntry& out, int& pix) {
  const float vx = p.x - x.x, vy = p.y - x.y, vz = p.z - x.z;
  const float r2 = vx * vx + vy * vy + vz * vz;
  if (!(r2 > 0.0f)) return false;
  const float r = sqrtf(r2);
  int k = hp_vec2pix_f32(a.nside, vx, vy, vz, hp_guard(a.nside, r));
  if (k < 0) {
    const double* x64 = origin64<kBucket>(a, si);
    k = hp_vec2pix_f64(a.nside, __dsub_rn(p64[0], x64[0]), __dsub_rn(p64[1], x64[1]),
                       __dsub_rn(p64[2], x64[2]));
  }
  float4 n = a.dirs[k];
  if constexpr (kBucket) {  // the directed beam (Sec. 3.4.1) points at its target
    const double* o = origin64<true>(a, si);
    if (int(o[7]) == k) n = make_float4(float(o[4]), float(o[5]), float(o[6]), n.w);
  }
  const float s = vx * n.x + vy * n.y + vz * n.z;
  if (!(s > 0.0f)) return false;
  out.s = s;
  out.rs = r / s;
  if constexpr (kBucket) {
    // the bucket walk keeps the projected distance in w; with the complex
    // source model (Sec. 2.7) a cell's source takes the beam only up to its
    // projected edge s - d, d its own ray back towards the bucket
    out.w = s;
    if constexpr (kCSM) {
      if (!(ref & kRefElement)) {
        const float d = a.csm_d[int64_t(ref) * a.npix + a.csm_anti[k]];
        out.s = fmaxf(s - d, 1e-30f);
      }
    }
  } else {
    out.w = (a.flags & TREVR2_SOFT) ? soft_kernel(r, a.hn[si]) : 1.0f / (kFourPi * r2);
  }
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

// Phase S for the sources whose running index is in [lo, lo + M): their
// references (a cell index, or an element index with kRefElement) go to
// U[].ref; make_sources then fills the records.  Returns the total number of
// sources of this receiver (warp-uniform).
template <bool kBucket = false, bool kPP = false>
static __device__ int phase_sources(const WalkArgs& a, float3 x, int si, int lane, int* stk, int cap,
                             SrcEntry* U, int* Up, int lo, float rpp = 0.0f) {
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
    if (q >= 0) {
      const NodeW nd = a.nodes[q];
      if (nd.meta & kMetaHasL) {
        if (!cell_opens<kBucket, kPP>(a, q, nd, x, si, rpp)) {
          emit_node = true;
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
      if (emit_node && idx >= 0 && idx < a.M) U[idx].ref = q;
      emitted += __popc(m);
    }
    // luminous elements of opened leaves
    int maxc = leaf_count;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) maxc = max(maxc, __shfl_xor_sync(0xffffffffu, maxc, o));
    for (int e = 0; e < maxc; ++e) {
      bool em = false;
      const int sj = leaf_first + e;
      if (e < leaf_count) em = a.pos32[sj].w > 0.0f && sj != si;
      const unsigned m = __ballot_sync(0xffffffffu, em);
      const int idx = emitted + __popc(m & lt) - lo;
      if (em && idx >= 0 && idx < a.M) U[idx].ref = sj | kRefElement;
      emitted += __popc(m);
    }
    __syncwarp();
  }
  return emitted;
}

// The records of the n staged sources, all lanes at once: beam, projected
// distance, r/s, kernel (make_source); a source the method skips (r = 0, or
// not in front of its beam) gets beam -1.
template <bool kBucket = false, bool kCSM = false>
static __device__ void make_sources(const WalkArgs& a, float3 x, int si, int lane, SrcEntry* U,
                                    int* Up, int n) {
  for (int e = lane; e < n; e += 32) {
    const int ref = U[e].ref;
    float3 p;
    const double* p64;
    if (ref & kRefElement) {
      const int64_t j = ref & 0x7fffffff;
      const float4 pj = a.pos32[j];
      p = make_float3(pj.x, pj.y, pj.z);
      p64 = a.pos64 + 3 * j;
    } else {
      const float4 c = a.csrc[ref];
      p = make_float3(c.x, c.y, c.z);
      p64 = a.c64 + 3 * int64_t(ref);
    }
    SrcEntry ent;
    int pix = -1;
    if (make_source<kBucket, kCSM>(a, p, p64, x, si, ref, ent, pix)) U[e] = ent; else pix = -1;
    Up[e] = pix;
  }
  __syncwarp();
}

// Bucket the n records of U by beam into V, skipping beam -1; off[k] ends as
// the end of bucket k (its start is off[k-1], or 0).  Each bucket is sorted
// by (s, source).  Returns the number of records binned.
static __device__ int bin_sources(const WalkArgs& a, int lane, SrcEntry* U, const int* Up, int n,
                                  SrcEntry* V, int* off) {
  const int npix = a.npix;
  for (int k = lane; k < npix; k += 32) off[k] = 0;
  __syncwarp();
  for (int e = lane; e < n; e += 32)
    if (Up[e] >= 0) atomicAdd(&off[Up[e]], 1);
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
    if (Up[e] < 0) continue;
    const int slot = atomicAdd(&off[Up[e]], 1);
    V[slot] = U[e];
  }
  __syncwarp();
  n = off[npix - 1];  // records binned
  // each record's rank in its bucket by (projected distance, source), all
  // lanes at once: the sorted buckets go to U, then back to V
  for (int e = lane; e < n; e += 32) {
    int lo = 0, hi = npix - 1;  // the bucket holding position e: first k with off[k] > e
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (off[mid] > e) hi = mid; else lo = mid + 1;
    }
    const int s0 = lo ? off[lo - 1] : 0, s1 = off[lo];
    const SrcEntry v = V[e];
    int r = 0;
    for (int j = s0; j < s1; ++j) {
      const SrcEntry w = V[j];
      r += (w.s < v.s) || (w.s == v.s && w.ref < v.ref);
    }
    U[s0 + r] = v;
  }
  __syncwarp();
  for (int e = lane; e < n; e += 32) V[e] = U[e];
  __syncwarp();
  return n;
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

template <int NBP>
__device__ __forceinline__ void store_bands(float* p, const BandVec<NBP>& v) {
  if constexpr (NBP == 4) {
    *reinterpret_cast<float4*>(p) = make_float4(v.v[0], v.v[1], v.v[2], v.v[3]);
  } else if constexpr (NBP == 2) {
    *reinterpret_cast<float2*>(p) = make_float2(v.v[0], v.v[1]);
  } else {
    *p = v.v[0];
  }
}

// The beams that hold sources, farthest source first (longest walks first,
// so that lanes finish together): a counting sort on 32 log-spaced buckets
// of the farthest source's distance.  Returns how many there are.
static __device__ int order_beams(const WalkArgs& a, int lane, const SrcEntry* V, const int* off,
                           int* order, int* cnt) {
  cnt[lane] = 0;
  __syncwarp();
  for (int k = lane; k < a.npix; k += 32) {
    const int s0 = k ? off[k - 1] : 0, s1 = off[k];
    if (s1 > s0) {
      const int b = min(31, max(0, int(-4.0f * __log2f(V[s1 - 1].s))));
      atomicAdd(&cnt[b], 1);
    }
  }
  __syncwarp();
  const int c = cnt[lane];
  const int incl = warp_incl_scan(c, lane);
  const int total = __shfl_sync(0xffffffffu, incl, 31);
  cnt[lane] = incl - c;
  __syncwarp();
  for (int k = lane; k < a.npix; k += 32) {
    const int s0 = k ? off[k - 1] : 0, s1 = off[k];
    if (s1 > s0) {
      const int b = min(31, max(0, int(-4.0f * __log2f(V[s1 - 1].s))));
      order[atomicAdd(&cnt[b], 1)] = k;
    }
  }
  __syncwarp();
  return total;
}

// ---------------------------------------------------------------------------
// Host side (walk.cu).
bool valid_nside(int nside);
// Per-tree walk arguments for one nside (everything but the receivers, the
// output and the buffers).
void fill_walk_args(const Tree* t, const Table* tb, int nside, float theta, const int* bsel,
                    int nbsel, uint32_t flags, int M, WalkArgs* a);
// Shared memory attribute and resident blocks per SM of a walk kernel.
int config_walk_kernel(const void* fn, int warps, size_t smem, int* per_sm, int* sms);
// Synchronises `st` and returns (and clears) the tree's device status.
int read_status(Tree* t, cudaStream_t st);

// Per-warp shared memory of a walk block: the traversal stacks, the beam
// bucket offsets, the beam order and its 32 bucket counts, the next-beam
// counter (padded to 16 bytes), the receiver's ancestor records.
inline size_t walk_smem(int warps, int stack_ints, int npix, int max_depth) {
  return size_t(warps) * (stack_ints + 2 * npix + 36 + 8 * (max_depth + 1)) * sizeof(int);
}

}  // namespace trevr2
