// Radiation tree build on the GPU (TREVR2, Sec. 2.3 and Sec. 2.6):
// FP64 normalisation + 63-bit Morton keys, a stable LSD radix sort,
// level-by-level bisection (a node splits while it holds more than `bucket`
// elements; empty halves become empty leaves), and a bottom-up pass for the
// summed luminosity per band, the centre of luminosity (one band-summed
// centre per cell), B = largest centre-to-corner distance (Sec. 2.5.2) and the
// bucket absorption sum(kappa m)/V_box (Sec. 2.6).  Sums run in FP64 and are
// rounded once to FP32 for the walk.
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <type_traits>
#include <string>

#include "internal.cuh"

namespace trevr2 {

// ---------------------------------------------------------------------------
// Errors
static thread_local char g_err[512];

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}
void clear_error() { g_err[0] = 0; }

static std::atomic<unsigned long long> g_launches{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

int cuda_fail(cudaError_t e, const char* what) {
  set_error("%s failed: %s", what, cudaGetErrorString(e));
  cudaGetLastError();
  return e == cudaErrorMemoryAllocation ? TREVR2_ENOMEM : TREVR2_ECUDA;
}

// ---------------------------------------------------------------------------
// Device allocations, and the failures a test can ask for (testing aids).
static std::atomic<int64_t> g_fail_alloc_after{-1};   // -1: off
static std::atomic<int> g_source_stack_cap{0};        // 0: off

// True for the one allocation a test asked to fail (then off again).
static bool injected_alloc_failure() {
  int64_t v = g_fail_alloc_after.load();
  while (v >= 0)
    if (g_fail_alloc_after.compare_exchange_weak(v, v - 1)) return v == 0;
  return false;
}

int device_alloc(void** p, size_t bytes, cudaStream_t st, const char* what) {
  *p = nullptr;
  if (injected_alloc_failure()) {
    set_error("%s of %zu bytes failed: out of memory (failure requested by "
              "trevr2_debug_set)", what, bytes);
    return TREVR2_ENOMEM;
  }
  cudaError_t e = cudaMallocAsync(p, bytes, st);
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    set_error("%s of %zu bytes failed: %s", what, bytes, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? TREVR2_ENOMEM : TREVR2_ECUDA;
  }
  return TREVR2_OK;
}

int debug_source_stack_cap() { return g_source_stack_cap.load(); }

// ---------------------------------------------------------------------------
// Exclusive scan (block scan of 2048 values + recursive scan of block sums).
constexpr int kScanThreads = 1024;
constexpr int kScanItems = 2 * kScanThreads;

__global__ void k_scan_block(int* d, int64_t n, int* block_sums) {
  __shared__ int s[kScanItems];
  const int64_t base = int64_t(blockIdx.x) * kScanItems;
  const int t = threadIdx.x;
  int64_t i0 = base + 2 * t, i1 = i0 + 1;
  int a = i0 < n ? d[i0] : 0;
  int b = i1 < n ? d[i1] : 0;
  s[2 * t] = a;
  s[2 * t + 1] = b;
  // Blelloch up-sweep / down-sweep
  int offset = 1;
  for (int w = kScanItems >> 1; w > 0; w >>= 1) {
    __syncthreads();
    if (t < w) {
      int ai = offset * (2 * t + 1) - 1, bi = offset * (2 * t + 2) - 1;
      s[bi] += s[ai];
    }
    offset <<= 1;
  }
  __syncthreads();
  if (t == 0) {
    if (block_sums) block_sums[blockIdx.x] = s[kScanItems - 1];
    s[kScanItems - 1] = 0;
  }
  for (int w = 1; w < kScanItems; w <<= 1) {
    offset >>= 1;
    __syncthreads();
    if (t < w) {
      int ai = offset * (2 * t + 1) - 1, bi = offset * (2 * t + 2) - 1;
      int tmp = s[ai];
      s[ai] = s[bi];
      s[bi] += tmp;
    }
  }
  __syncthreads();
  if (i0 < n) d[i0] = s[2 * t];
  if (i1 < n) d[i1] = s[2 * t + 1];
}

__global__ void k_scan_add(int* d, int64_t n, const int* block_offsets) {
  const int64_t base = int64_t(blockIdx.x) * kScanItems;
  int add = block_offsets[blockIdx.x];
  for (int k = threadIdx.x; k < kScanItems; k += blockDim.x) {
    int64_t i = base + k;
    if (i < n) d[i] += add;
  }
}

__global__ void k_scan_total(const int* scanned, const int* orig_last, int64_t n, int* total) {
  *total = n ? scanned[n - 1] + *orig_last : 0;
}

__global__ void k_copy_last(const int* d, int64_t n, int* out) { *out = n ? d[n - 1] : 0; }

size_t scan_ws_ints(int64_t n) {
  const int64_t nblocks = (n + kScanItems - 1) / kScanItems;
  return 1 + (nblocks > 1 ? size_t(nblocks) + scan_ws_ints(nblocks) : 0);
}

// ws: the last input value, then the block sums of each recursion level.
static int scan_with_ws(int* d, int64_t n, int* d_total, cudaStream_t st, int* ws) {
  int* last = ws;
  k_copy_last<<<1, 1, 0, st>>>(d, n, last); note_launch();
  if (n > 0) {
    int64_t nblocks = (n + kScanItems - 1) / kScanItems;
    if (nblocks == 1) {
      k_scan_block<<<1, kScanThreads, 0, st>>>(d, n, nullptr); note_launch();
    } else {
      int* sums = ws + 1;
      k_scan_block<<<unsigned(nblocks), kScanThreads, 0, st>>>(d, n, sums); note_launch();
      T2_CHECK(scan_with_ws(sums, nblocks, nullptr, st, sums + nblocks));
      k_scan_add<<<unsigned(nblocks), 256, 0, st>>>(d, n, sums); note_launch();
    }
  }
  if (d_total) k_scan_total<<<1, 1, 0, st>>>(d, last, n, d_total); note_launch();
  T2_CUDA(cudaGetLastError());
  return TREVR2_OK;
}

int scan_exclusive_i32(int* d, int64_t n, int* d_total, cudaStream_t st, int* ws) {
  if (ws) return scan_with_ws(d, n, d_total, st, ws);
  T2_CHECK(dalloc(&ws, scan_ws_ints(n), st));
  const int rc = scan_with_ws(d, n, d_total, st, ws);
  dfree(ws, st);
  return rc;
}

// ---------------------------------------------------------------------------
// Stable LSD radix sort, 8 bits per pass.  Each tile of 2048 keys is ranked
// in 8 rounds of 256 keys; inside a round, warps rank their lanes with
// __match_any_sync and a per-warp digit count, so equal digits keep their
// input order (stability gives the (key, caller index) order).
constexpr int kSortThreads = 256;
constexpr int kSortTile = 2048;
constexpr int kSortWarps = kSortThreads / 32;

__global__ void k_radix_hist(const uint64_t* __restrict__ keys, int64_t n, int shift,
                             int* __restrict__ hist, int ntiles) {
  __shared__ int h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = int64_t(blockIdx.x) * kSortTile;
  for (int k = threadIdx.x; k < kSortTile; k += kSortThreads) {
    int64_t i = base + k;
    if (i < n) atomicAdd(&h[(keys[i] >> shift) & 255u], 1);
  }
  __syncthreads();
  hist[int64_t(threadIdx.x) * ntiles + blockIdx.x] = h[threadIdx.x];
}

__global__ void k_radix_scatter(const uint64_t* __restrict__ kin, const int* __restrict__ vin,
                                uint64_t* __restrict__ kout, int* __restrict__ vout, int64_t n,
                                int shift, const int* __restrict__ offsets, int ntiles) {
  __shared__ int base[256];
  __shared__ int wh[kSortWarps][256];
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  base[t] = offsets[int64_t(t) * ntiles + blockIdx.x];
  const unsigned lt_mask = (1u << lane) - 1u;
  const int64_t tile0 = int64_t(blockIdx.x) * kSortTile;
  for (int round = 0; round < kSortTile / kSortThreads; ++round) {
    for (int w = 0; w < kSortWarps; ++w) wh[w][t] = 0;
    __syncthreads();
    int64_t i = tile0 + round * kSortThreads + t;
    bool valid = i < n;
    uint64_t key = valid ? kin[i] : 0;
    int val = valid ? vin[i] : 0;
    int digit = valid ? int((key >> shift) & 255u) : 256;
    unsigned peers = __match_any_sync(0xffffffffu, digit);
    int intra = __popc(peers & lt_mask);
    if (valid && intra == 0) wh[warp][digit] = __popc(peers);
    __syncthreads();
    {
      int run = base[t];
      for (int w = 0; w < kSortWarps; ++w) {
        int c = wh[w][t];
        wh[w][t] = run;
        run += c;
      }
      base[t] = run;
    }
    __syncthreads();
    if (valid) {
      int dst = wh[warp][digit] + intra;
      kout[dst] = key;
      vout[dst] = val;
    }
    __syncthreads();
  }
}

size_t radix_ws_bytes(int64_t n) {
  const int64_t ntiles = (n + kSortTile - 1) / kSortTile;
  auto up = [](size_t b) { return (b + 255) & ~size_t(255); };
  return up(sizeof(uint64_t) * size_t(n)) + up(sizeof(int) * size_t(n)) +
         up(sizeof(int) * 256 * size_t(ntiles)) + up(sizeof(int) * scan_ws_ints(256 * ntiles));
}

int radix_sort_u64_i32(uint64_t* keys, int* vals, int64_t n, cudaStream_t st, int key_bits,
                       void* ws) {
  if (n <= 1) return TREVR2_OK;
  // an even number of 8-bit passes, so the result ends in the caller's buffers
  int passes = (std::min(std::max(key_bits, 1), 64) + 7) / 8;
  passes += passes & 1;
  const int ntiles = int((n + kSortTile - 1) / kSortTile);
  const bool own = ws == nullptr;
  if (own) T2_CHECK(device_alloc(&ws, radix_ws_bytes(n), st, "sort workspace"));
  auto up = [](size_t b) { return (b + 255) & ~size_t(255); };
  char* p = static_cast<char*>(ws);
  uint64_t* k2 = reinterpret_cast<uint64_t*>(p);
  p += up(sizeof(uint64_t) * size_t(n));
  int* v2 = reinterpret_cast<int*>(p);
  p += up(sizeof(int) * size_t(n));
  int* hist = reinterpret_cast<int*>(p);
  p += up(sizeof(int) * 256 * size_t(ntiles));
  int* scan_ws = reinterpret_cast<int*>(p);
  uint64_t *ka = keys, *kb = k2;
  int *va = vals, *vb = v2;
  int rc = TREVR2_OK;
  for (int shift = 0; shift < 8 * passes && rc == TREVR2_OK; shift += 8) {
    k_radix_hist<<<ntiles, kSortThreads, 0, st>>>(ka, n, shift, hist, ntiles); note_launch();
    rc = scan_exclusive_i32(hist, int64_t(256) * ntiles, nullptr, st, scan_ws);
    if (rc != TREVR2_OK) break;
    k_radix_scatter<<<ntiles, kSortThreads, 0, st>>>(ka, va, kb, vb, n, shift, hist, ntiles); note_launch();
    std::swap(ka, kb);
    std::swap(va, vb);
  }
  if (own) cudaFreeAsync(ws, st);
  if (rc != TREVR2_OK) return rc;
  T2_CUDA(cudaGetLastError());
  return TREVR2_OK;
}

// ---------------------------------------------------------------------------
// Input validation and bounds.
__global__ void k_validate(const double* __restrict__ pos, const float* __restrict__ mass,
                           const float* __restrict__ kappa, const float* __restrict__ lum,
                           const float* __restrict__ h, int64_t N, int nb,
                           double* __restrict__ partial /*[grid][6]*/, uint32_t* status) {
  __shared__ double smin[3][256], smax[3][256];
  double mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
  bool bad = false;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < N;
       i += int64_t(gridDim.x) * blockDim.x) {
    for (int a = 0; a < 3; ++a) {
      double x = pos[3 * i + a];
      bad |= !isfinite(x);
      mn[a] = fmin(mn[a], x);
      mx[a] = fmax(mx[a], x);
    }
    float m = mass[i];
    bad |= !(m >= 0.0f) || !isfinite(m);
    if (h) bad |= !(h[i] > 0.0f) || !isfinite(h[i]);
    for (int b = 0; b < nb; ++b) {
      float k = kappa[i * nb + b], l = lum[i * nb + b];
      bad |= !(k >= 0.0f) || !isfinite(k) || !(l >= 0.0f) || !isfinite(l);
    }
  }
  if (bad) atomicOr(status, kStatusBadInput);
  for (int a = 0; a < 3; ++a) {
    smin[a][threadIdx.x] = mn[a];
    smax[a][threadIdx.x] = mx[a];
  }
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
      for (int a = 0; a < 3; ++a) {
        smin[a][threadIdx.x] = fmin(smin[a][threadIdx.x], smin[a][threadIdx.x + w]);
        smax[a][threadIdx.x] = fmax(smax[a][threadIdx.x], smax[a][threadIdx.x + w]);
      }
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int a = 0; a < 3; ++a) {
      partial[6 * blockIdx.x + a] = smin[a][0];
      partial[6 * blockIdx.x + 3 + a] = smax[a][0];
    }
}

// Sec. 2.3: normalise in FP64 and interleave the 21-bit cell indices,
// bit 62 = x MSB, then y, then z.
__device__ inline uint64_t spread3(uint64_t v) {
  v &= 0x1fffffull;
  v = (v | (v << 32)) & 0x1f00000000ffffull;
  v = (v | (v << 16)) & 0x1f0000ff0000ffull;
  v = (v | (v << 8)) & 0x100f00f00f00f00full;
  v = (v | (v << 4)) & 0x10c30c30c30c30c3ull;
  v = (v | (v << 2)) & 0x1249249249249249ull;
  return v;
}

__global__ void k_morton(const double* __restrict__ pos, int64_t N, double lo0, double lo1,
                         double lo2, double size, uint64_t* __restrict__ keys,
                         int* __restrict__ vals) {
  int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (i >= N) return;
  const double lo[3] = {lo0, lo1, lo2};
  uint64_t k[3];
  for (int a = 0; a < 3; ++a) {
    double u = __ddiv_rn(__dsub_rn(pos[3 * i + a], lo[a]), size);
    double f = floor(__dmul_rn(u, 2097152.0));
    f = fmin(fmax(f, 0.0), 2097151.0);
    k[a] = uint64_t(f);
  }
  keys[i] = (spread3(k[0]) << 2) | (spread3(k[1]) << 1) | spread3(k[2]);
  vals[i] = int(i);
}

// Sorted element data used by the walk.
__global__ void k_gather_elements(const double* __restrict__ pos, const float* __restrict__ mass,
                                  const float* __restrict__ kappa, const float* __restrict__ lum,
                                  const float* __restrict__ h, const int* __restrict__ perm,
                                  int64_t N, int nb, int nbp, double lo0, double lo1, double lo2,
                                  double size, float h_default, int* __restrict__ inv,
                                  double* __restrict__ pos64, float4* __restrict__ pos32,
                                  float* __restrict__ Lelem, float* __restrict__ km,
                                  float* __restrict__ hn, float* __restrict__ ms) {
  int64_t s = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (s >= N) return;
  int i = perm[s];
  inv[i] = int(s);
  const double lo[3] = {lo0, lo1, lo2};
  double u[3];
  for (int a = 0; a < 3; ++a) {
    u[a] = __ddiv_rn(__dsub_rn(pos[3 * int64_t(i) + a], lo[a]), size);
    pos64[3 * s + a] = u[a];
  }
  double lt = 0.0;
  for (int b = 0; b < nbp; ++b) {
    float l = b < nb ? lum[int64_t(i) * nb + b] : 0.0f;
    float k = b < nb ? kappa[int64_t(i) * nb + b] : 0.0f;
    Lelem[s * nbp + b] = l;
    km[s * nbp + b] = k * mass[i];
    lt = __dadd_rn(lt, double(l));
  }
  pos32[s] = make_float4(float(u[0]), float(u[1]), float(u[2]), float(lt));
  float hh = h ? h[i] : h_default;
  hn[s] = float(double(hh) / size);
  ms[s] = mass[i];
}

// ---------------------------------------------------------------------------
// Level-by-level bisection.
__global__ void k_split_mark(const uint64_t* __restrict__ keys, int64_t lb, int64_t le, int bucket,
                             const int* __restrict__ depth, const int* __restrict__ first,
                             const int* __restrict__ count, int* __restrict__ flag,
                             int* __restrict__ mid) {
  int64_t q = lb + blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (q >= le) return;
  int d = depth[q], c = count[q], f = first[q];
  bool split = c > bucket && d < kMaxDepth;
  flag[q - lb] = split ? 1 : 0;
  if (!split) return;
  // keys in [f, f+c) share the node's prefix, so bit (62 - d) is monotone
  const int bit = kMaxDepth - 1 - d;
  int lo = f, hi = f + c;  // first index with the bit set
  while (lo < hi) {
    int m = lo + ((hi - lo) >> 1);
    if ((keys[m] >> bit) & 1ull) hi = m; else lo = m + 1;
  }
  mid[q - lb] = lo;
}

__global__ void k_split_emit(int64_t lb, int64_t le, int64_t child_base,
                             const int* __restrict__ flag_scan, const int* __restrict__ flag,
                             const int* __restrict__ mid, uint64_t* __restrict__ prefix,
                             int* __restrict__ depth, int* __restrict__ first,
                             int* __restrict__ count, int* __restrict__ child,
                             int* __restrict__ parent) {
  int64_t q = lb + blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (q >= le) return;
  int64_t j = q - lb;
  if (!flag[j]) {
    child[q] = -1;
    return;
  }
  int64_t c = child_base + 2 * int64_t(flag_scan[j]);
  child[q] = int(c);
  int d = depth[q], f = first[q], n = count[q], m = mid[j];
  uint64_t p = prefix[q];
  const int bit = kMaxDepth - 1 - d;
  prefix[c] = p;
  prefix[c + 1] = p | (1ull << bit);
  depth[c] = depth[c + 1] = d + 1;
  first[c] = f;
  count[c] = m - f;
  first[c + 1] = m;
  count[c + 1] = f + n - m;
  parent[c] = parent[c + 1] = int(q);
  child[c] = child[c + 1] = -1;
}

__global__ void k_leaf_flags(const int* __restrict__ child, int64_t n, int* __restrict__ out) {
  int64_t q = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (q < n) out[q] = child[q] >= 0 ? 1 : 0;
}

__global__ void k_finish_int_index(const int* __restrict__ child, int64_t n, int* __restrict__ idx) {
  int64_t q = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (q < n && child[q] < 0) idx[q] = -1;
}

// ---------------------------------------------------------------------------
// Bottom-up aggregates for one depth (children are done before parents).
__device__ inline void node_box_norm(uint64_t prefix, int depth, double lo[3], double ext[3]) {
  for (int a = 0; a < 3; ++a) {
    uint64_t k = 0;
    for (int l = 0; l < kKeyBits; ++l) k = (k << 1) | ((prefix >> (3 * (kKeyBits - 1 - l) + 2 - a)) & 1ull);
    lo[a] = double(k) * (1.0 / 2097152.0);
    ext[a] = ldexp(1.0, -splits_on_axis(depth, a));
  }
}

__global__ void k_aggregate_level(int64_t lb, int64_t le, int nb, int nbp, double inv_size2,
                                  const uint64_t* __restrict__ prefix, const int* __restrict__ depth,
                                  const int* __restrict__ first, const int* __restrict__ count,
                                  const int* __restrict__ child, const int* __restrict__ int_index,
                                  const double* __restrict__ pos64, const float* __restrict__ Lelem,
                                  const int* __restrict__ perm, const float* __restrict__ kappa,
                                  const float* __restrict__ mass, double* __restrict__ L64,
                                  double* __restrict__ cs64 /*[n][4]: sum Lt x, sum Lt*/,
                                  uint32_t* __restrict__ flags64, float* __restrict__ Lnode,
                                  float4* __restrict__ csrc, double* __restrict__ c64,
                                  double* __restrict__ B64, float* __restrict__ alpha_leaf,
                                  NodeW* __restrict__ nodes) {
  int64_t q = lb + blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (q >= le) return;
  const int d = depth[q];
  double lo[3], ext[3];
  node_box_norm(prefix[q], d, lo, ext);
  const int c = child[q];
  double cs[4] = {0, 0, 0, 0};
  uint32_t has = 0;
  if (c < 0) {
    const int f = first[q], n = count[q];
    double Lb[4] = {0, 0, 0, 0}, kmb[4] = {0, 0, 0, 0};
    for (int e = f; e < f + n; ++e) {
      double lt = 0.0;
      for (int b = 0; b < nb; ++b) {
        double l = double(Lelem[int64_t(e) * nbp + b]);
        Lb[b] = __dadd_rn(Lb[b], l);
        lt = __dadd_rn(lt, l);
        // kappa and m are float32: their FP64 product is exact
        const int i = perm[e];
        kmb[b] = __dadd_rn(kmb[b], __dmul_rn(double(kappa[int64_t(i) * nb + b]), double(mass[i])));
      }
      for (int a = 0; a < 3; ++a) cs[a] = __dadd_rn(cs[a], __dmul_rn(lt, pos64[3 * int64_t(e) + a]));
      cs[3] = __dadd_rn(cs[3], lt);
    }
    const double V = ext[0] * ext[1] * ext[2];  // exact powers of two
    for (int b = 0; b < nbp; ++b) {
      double al = b < nb ? kmb[b] / V * inv_size2 : 0.0;
      alpha_leaf[q * nbp + b] = float(al);
      if (al > 0.0) has |= kMetaHasAlpha;
    }
    for (int b = 0; b < 4; ++b) L64[q * 4 + b] = b < nb ? Lb[b] : 0.0;
  } else {
    for (int b = 0; b < 4; ++b) L64[q * 4 + b] = __dadd_rn(L64[int64_t(c) * 4 + b], L64[int64_t(c + 1) * 4 + b]);
    for (int a = 0; a < 4; ++a) cs[a] = __dadd_rn(cs64[int64_t(c) * 4 + a], cs64[int64_t(c + 1) * 4 + a]);
    has = (flags64[c] | flags64[c + 1]) & kMetaHasAlpha;
    for (int b = 0; b < nbp; ++b) alpha_leaf[q * nbp + b] = 0.0f;
  }
  for (int a = 0; a < 4; ++a) cs64[q * 4 + a] = cs[a];
  double cc[3];
  for (int a = 0; a < 3; ++a) cc[a] = cs[3] > 0.0 ? cs[a] / cs[3] : lo[a] + 0.5 * ext[a];
  if (cs[3] > 0.0) has |= kMetaHasL;
  flags64[q] = has;
  // B: farthest box corner from the centre of luminosity (Sec. 2.5.2)
  double B2 = 0.0;
  for (int corner = 0; corner < 8; ++corner) {
    double r2 = 0.0;
    for (int a = 0; a < 3; ++a) {
      double p = ((corner >> a) & 1) ? lo[a] + ext[a] : lo[a];
      double dd = __dsub_rn(p, cc[a]);
      r2 = __dadd_rn(r2, __dmul_rn(dd, dd));
    }
    B2 = fmax(B2, r2);
  }
  double B = sqrt(B2);
  for (int a = 0; a < 3; ++a) c64[3 * q + a] = cc[a];
  B64[q] = B;
  for (int b = 0; b < nbp; ++b) Lnode[q * nbp + b] = float(L64[q * 4 + b]);
  csrc[q] = make_float4(float(cc[0]), float(cc[1]), float(cc[2]), float(cs[3]));
  NodeW w;
  w.lo[0] = float(lo[0]);
  w.lo[1] = float(lo[1]);
  w.lo[2] = float(lo[2]);
  w.B = float(B);
  w.child = c;
  w.aux = c < 0 ? first[q] : int_index[q];
  w.count = count[q];
  w.meta = uint32_t(d) | (uint32_t(d % 3) << kMetaAxisShift) | (c < 0 ? kMetaLeaf : 0u) | has;
  if (c >= 0) {
    if (flags64[c] & kMetaHasAlpha) w.meta |= kMetaChild0Alpha;
    if (flags64[c + 1] & kMetaHasAlpha) w.meta |= kMetaChild1Alpha;
  }
  nodes[q] = w;
}

// ---------------------------------------------------------------------------
static int grow(Tree* t, int64_t need, int64_t& cap, cudaStream_t st) {
  if (need <= cap) return TREVR2_OK;
  int64_t ncap = std::max<int64_t>(cap, 1024);
  while (ncap < need) ncap *= 2;
  auto regrow = [&](auto*& p) -> int {
    using T = std::remove_pointer_t<std::remove_reference_t<decltype(p)>>;
    T* q = nullptr;
    int rc = dalloc(&q, ncap, st);
    if (rc) return rc;
    if (p) {
      cudaError_t e = cudaMemcpyAsync(q, p, cap * sizeof(T), cudaMemcpyDeviceToDevice, st);
      if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync");
      dfree(p, st);
    }
    p = q;
    return TREVR2_OK;
  };
  T2_CHECK(regrow(t->prefix));
  T2_CHECK(regrow(t->depth));
  T2_CHECK(regrow(t->first));
  T2_CHECK(regrow(t->count));
  T2_CHECK(regrow(t->child));
  T2_CHECK(regrow(t->parent));
  cap = ncap;
  return TREVR2_OK;
}

__global__ void k_init_root(int64_t N, uint64_t* prefix, int* depth, int* first, int* count,
                            int* child, int* parent) {
  prefix[0] = 0;
  depth[0] = 0;
  first[0] = 0;
  count[0] = int(N);
  child[0] = -1;
  parent[0] = -1;
}

static void free_tree(Tree* t, cudaStream_t st) {
  dfree(t->keys, st);
  dfree(t->perm, st);
  dfree(t->inv, st);
  dfree(t->pos64, st);
  dfree(t->pos32, st);
  dfree(t->Lelem, st);
  dfree(t->km, st);
  dfree(t->mass, st);
  dfree(t->hn, st);
  dfree(t->prefix, st);
  dfree(t->depth, st);
  dfree(t->first, st);
  dfree(t->count, st);
  dfree(t->child, st);
  dfree(t->parent, st);
  dfree(t->int_index, st);
  dfree(t->nodes, st);
  dfree(t->Lnode, st);
  dfree(t->csrc, st);
  dfree(t->c64, st);
  dfree(t->B64, st);
  dfree(t->alpha_leaf, st);
  dfree(t->dtau, st);
  dfree(t->nodes_refined, st);
  for (Table& tb : t->tables) {
    dfree(tb.alpha, st);
    dfree(tb.dirs, st);
    dfree(tb.dirs64, st);
    dfree(tb.geo, st);
    dfree(tb.csm_tau, st);
    dfree(tb.csm_d, st);
    dfree(tb.csm_anti, st);
  }
  t->tables.clear();
  if (t->scratch) cudaFreeAsync(t->scratch, st);
  t->scratch = nullptr;
  if (t->order_buf) cudaFreeAsync(t->order_buf, st);
  t->order_buf = nullptr;
  dfree(t->status, st);
  dfree(t->counter, st);
}

static inline unsigned blocks_for(int64_t n, int threads) {
  return unsigned((n + threads - 1) / threads);
}

static int build_impl(Tree* t, const double* pos, const float* mass, const float* kappa,
                      const float* lum, const float* h, const double* box_lo, double box_size,
                      cudaStream_t st) {
  const int64_t N = t->N;
  const int nb = t->nb, nbp = t->nbp;
  T2_CHECK(dalloc(&t->status, 1, st));
  T2_CHECK(dalloc(&t->counter, 1, st));
  T2_CUDA(cudaMemsetAsync(t->status, 0, sizeof(uint32_t), st));

  // 1. validation and bounding box
  const int vthreads = 256;
  const int vblocks = int(std::min<int64_t>(std::max<int64_t>(blocks_for(N, vthreads), 1), 1024));
  DeviceTemp<double> partial(st);
  T2_CHECK(dalloc(&partial.p, size_t(vblocks) * 6, st));
  if (N > 0)
    k_validate<<<vblocks, vthreads, 0, st>>>(pos, mass, kappa, lum, h, N, nb, partial.p, t->status); note_launch();
  std::vector<double> hpart(size_t(vblocks) * 6);
  uint32_t hstatus = 0;
  if (N > 0) {
    T2_CUDA(cudaMemcpyAsync(hpart.data(), partial.p, hpart.size() * sizeof(double),
                            cudaMemcpyDeviceToHost, st));
    T2_CUDA(cudaMemcpyAsync(&hstatus, t->status, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
  }
  T2_CUDA(cudaStreamSynchronize(st));
  dfree(partial.p, st);
  if (hstatus & kStatusBadInput) {
    set_error("trevr2_build: non-finite position, or negative/non-finite mass, kappa, lum or h");
    return TREVR2_EINVAL;
  }
  double mn[3] = {0, 0, 0}, mx[3] = {0, 0, 0};
  if (N > 0) {
    for (int a = 0; a < 3; ++a) {
      mn[a] = INFINITY;
      mx[a] = -INFINITY;
    }
    for (int b = 0; b < vblocks; ++b)
      for (int a = 0; a < 3; ++a) {
        mn[a] = std::min(mn[a], hpart[6 * b + a]);
        mx[a] = std::max(mx[a], hpart[6 * b + 3 + a]);
      }
  }
  if (box_lo && box_size > 0.0) {
    for (int a = 0; a < 3; ++a) t->lo[a] = box_lo[a];
    t->size = box_size;
    if (N > 0)
      for (int a = 0; a < 3; ++a)
        if (mn[a] < box_lo[a] || mx[a] > box_lo[a] + box_size) {
          set_error("trevr2_build: a position lies outside the given root cube");
          return TREVR2_EINVAL;
        }
  } else {
    double ext = 0.0;
    for (int a = 0; a < 3; ++a) {
      t->lo[a] = mn[a];
      ext = std::max(ext, mx[a] - mn[a]);
    }
    t->size = ext > 0.0 ? ext : 1.0;
  }

  // 2. keys and stable sort
  T2_CHECK(dalloc(&t->keys, N, st));
  T2_CHECK(dalloc(&t->perm, N, st));
  if (N > 0)
    k_morton<<<blocks_for(N, 256), 256, 0, st>>>(pos, N, t->lo[0], t->lo[1], t->lo[2], t->size,
                                                 t->keys, t->perm); note_launch();
  T2_CHECK(radix_sort_u64_i32(t->keys, t->perm, N, st));

  // 3. sorted element data
  int64_t ngas = 0;  // h default: (V_root / N_gas)^(1/3), counted on the host only if needed
  float h_default = 1.0f;
  if (!h && N > 0) {
    std::vector<float> hm(N);
    T2_CUDA(cudaMemcpyAsync(hm.data(), mass, N * sizeof(float), cudaMemcpyDeviceToHost, st));
    T2_CUDA(cudaStreamSynchronize(st));
    for (float m : hm) ngas += m > 0.0f;
    h_default = float(std::cbrt(t->size * t->size * t->size / double(std::max<int64_t>(ngas, 1))));
  }
  T2_CHECK(dalloc(&t->inv, N, st));
  T2_CHECK(dalloc(&t->pos64, 3 * N, st));
  T2_CHECK(dalloc(&t->pos32, N, st));
  T2_CHECK(dalloc(&t->Lelem, N * nbp, st));
  T2_CHECK(dalloc(&t->km, N * nbp, st));
  T2_CHECK(dalloc(&t->hn, N, st));
  T2_CHECK(dalloc(&t->mass, N, st));
  if (N > 0)
    k_gather_elements<<<blocks_for(N, 256), 256, 0, st>>>(
        pos, mass, kappa, lum, h, t->perm, N, nb, nbp, t->lo[0], t->lo[1], t->lo[2], t->size,
        h_default, t->inv, t->pos64, t->pos32, t->Lelem, t->km, t->hn, t->mass); note_launch();

  // 4. bisection, one depth at a time
  int64_t cap = 0;
  T2_CHECK(grow(t, std::max<int64_t>(1024, 4 * (N / std::max(t->bucket, 1)) + 64), cap, st));
  k_init_root<<<1, 1, 0, st>>>(N, t->prefix, t->depth, t->first, t->count, t->child, t->parent); note_launch();
  DeviceTemp<int> flag_t(st), fscan_t(st), mid_t(st), dtotal_t(st);
  int*& flag = flag_t.p;
  int*& fscan = fscan_t.p;
  int*& mid = mid_t.p;
  int*& dtotal = dtotal_t.p;
  int64_t flag_cap = 1024;
  T2_CHECK(dalloc(&flag, flag_cap, st));
  T2_CHECK(dalloc(&fscan, flag_cap, st));
  T2_CHECK(dalloc(&mid, flag_cap, st));
  T2_CHECK(dalloc(&dtotal, 1, st));
  t->level_begin.assign(1, 0);
  int64_t lb = 0, le = 1;
  int level = 0;
  for (;;) {
    const int64_t m = le - lb;
    if (m > flag_cap) {
      dfree(flag, st);
      dfree(fscan, st);
      dfree(mid, st);
      while (flag_cap < m) flag_cap *= 2;
      T2_CHECK(dalloc(&flag, flag_cap, st));
      T2_CHECK(dalloc(&fscan, flag_cap, st));
      T2_CHECK(dalloc(&mid, flag_cap, st));
    }
    k_split_mark<<<blocks_for(m, 256), 256, 0, st>>>(t->keys, lb, le, t->bucket, t->depth,
                                                      t->first, t->count, flag, mid); note_launch();
    T2_CUDA(cudaMemcpyAsync(fscan, flag, m * sizeof(int), cudaMemcpyDeviceToDevice, st));
    T2_CHECK(scan_exclusive_i32(fscan, m, dtotal, st));
    int total = 0;
    T2_CUDA(cudaMemcpyAsync(&total, dtotal, sizeof(int), cudaMemcpyDeviceToHost, st));
    T2_CUDA(cudaStreamSynchronize(st));
    if (le + 2 * int64_t(total) > (int64_t(1) << 31) - 1) {
      set_error("trevr2_build: more than 2^31 nodes");
      return TREVR2_EUNSUPPORTED;
    }
    T2_CHECK(grow(t, le + 2 * int64_t(total), cap, st));
    k_split_emit<<<blocks_for(m, 256), 256, 0, st>>>(lb, le, le, fscan, flag, mid, t->prefix,
                                                      t->depth, t->first, t->count, t->child,
                                                      t->parent); note_launch();
    t->level_begin.push_back(le);
    if (total == 0) break;
    lb = le;
    le += 2 * int64_t(total);
    ++level;
  }
  t->n_nodes = le;
  t->max_depth = level;
  dfree(flag, st);
  dfree(fscan, st);
  dfree(mid, st);

  // internal-node rows of the alpha tables
  const int64_t n = t->n_nodes;
  T2_CHECK(dalloc(&t->int_index, n, st));
  k_leaf_flags<<<blocks_for(n, 256), 256, 0, st>>>(t->child, n, t->int_index); note_launch();
  T2_CHECK(scan_exclusive_i32(t->int_index, n, dtotal, st));
  int nint = 0;
  T2_CUDA(cudaMemcpyAsync(&nint, dtotal, sizeof(int), cudaMemcpyDeviceToHost, st));
  k_finish_int_index<<<blocks_for(n, 256), 256, 0, st>>>(t->child, n, t->int_index); note_launch();
  dfree(dtotal, st);

  // 5. aggregates, deepest depth first
  T2_CHECK(dalloc(&t->nodes, n, st));
  T2_CHECK(dalloc(&t->Lnode, n * nbp, st));
  T2_CHECK(dalloc(&t->csrc, n, st));
  T2_CHECK(dalloc(&t->c64, 3 * n, st));
  T2_CHECK(dalloc(&t->B64, n, st));
  T2_CHECK(dalloc(&t->alpha_leaf, n * nbp, st));
  DeviceTemp<double> L64_t(st), cs64_t(st);
  DeviceTemp<uint32_t> fl_t(st);
  double*& L64 = L64_t.p;
  double*& cs64 = cs64_t.p;
  uint32_t*& fl = fl_t.p;
  T2_CHECK(dalloc(&L64, 4 * n, st));
  T2_CHECK(dalloc(&cs64, 4 * n, st));
  T2_CHECK(dalloc(&fl, n, st));
  const double inv_size2 = 1.0 / (t->size * t->size);
  for (int d = t->max_depth; d >= 0; --d) {
    int64_t a = t->level_begin[d], b = t->level_begin[d + 1];
    k_aggregate_level<<<blocks_for(b - a, 128), 128, 0, st>>>(
        a, b, nb, nbp, inv_size2, t->prefix, t->depth, t->first, t->count, t->child,
        t->int_index, t->pos64, t->Lelem, t->perm, kappa, mass, L64, cs64, fl, t->Lnode, t->csrc, t->c64,
        t->B64, t->alpha_leaf, t->nodes); note_launch();
  }
  dfree(L64, st);
  dfree(cs64, st);
  dfree(fl, st);
  T2_CUDA(cudaGetLastError());
  T2_CUDA(cudaStreamSynchronize(st));
  t->n_internal = nint;
  return TREVR2_OK;
}

}  // namespace trevr2

using namespace trevr2;

extern "C" {

const char* trevr2_last_error(void) { return g_err; }

int trevr2_debug_set(int what, int64_t value) {
  clear_error();
  switch (what) {
    case TREVR2_DEBUG_FAIL_ALLOC:
      if (value < -1) break;
      g_fail_alloc_after.store(value);
      return TREVR2_OK;
    case TREVR2_DEBUG_SOURCE_STACK:
      if (value < 0 || value > (int64_t(1) << 30)) break;
      g_source_stack_cap.store(int(value));
      return TREVR2_OK;
    default:
      break;
  }
  set_error("trevr2_debug_set: unknown setting %d or value %lld out of range", what,
            static_cast<long long>(value));
  return TREVR2_EINVAL;
}

int trevr2_debug_pool_used(uint64_t* bytes) {
  clear_error();
  if (!bytes) {
    set_error("trevr2_debug_pool_used: bytes is NULL");
    return TREVR2_EINVAL;
  }
  int dev = 0;
  T2_CUDA(cudaGetDevice(&dev));
  T2_CUDA(cudaDeviceSynchronize());
  cudaMemPool_t pool;
  T2_CUDA(cudaDeviceGetDefaultMemPool(&pool, dev));
  uint64_t used = 0;
  T2_CUDA(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used));
  *bytes = uint64_t(used);
  return TREVR2_OK;
}

uint64_t trevr2_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

int trevr2_build(const double* pos, const float* mass, const float* kappa, const float* lum,
                 const float* h, int64_t N, int nb, const double* box_lo, double box_size,
                 int bucket, void* stream, trevr2_tree** out) {
  clear_error();
  if (!out) {
    set_error("trevr2_build: out is NULL");
    return TREVR2_EINVAL;
  }
  *out = nullptr;
  if (N < 0 || (N > 0 && (!pos || !mass || !kappa || !lum))) {
    set_error("trevr2_build: N < 0 or a NULL input array");
    return TREVR2_EINVAL;
  }
  if (N >= (int64_t(1) << 31)) {
    set_error("trevr2_build: N must be below 2^31");
    return TREVR2_EUNSUPPORTED;
  }
  if (nb < 1 || nb > TREVR2_MAX_BANDS) {
    set_error("trevr2_build: nb = %d outside [1, %d]", nb, TREVR2_MAX_BANDS);
    return nb < 1 ? TREVR2_EINVAL : TREVR2_EUNSUPPORTED;
  }
  if (bucket < 1 || bucket > 4096) {
    set_error("trevr2_build: bucket = %d outside [1, 4096]", bucket);
    return TREVR2_EINVAL;
  }
  if (box_lo && box_size > 0.0) {
    for (int a = 0; a < 3; ++a)
      if (!std::isfinite(box_lo[a])) {
        set_error("trevr2_build: non-finite box_lo");
        return TREVR2_EINVAL;
      }
    if (!std::isfinite(box_size)) {
      set_error("trevr2_build: non-finite box_size");
      return TREVR2_EINVAL;
    }
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Tree* t = new (std::nothrow) Tree();
  if (!t) {
    set_error("trevr2_build: host allocation failed");
    return TREVR2_ENOMEM;
  }
  t->N = N;
  t->nb = nb;
  t->nbp = nbp_of(nb);
  t->bucket = bucket;
  t->has_h = h != nullptr;
  t->last_stream = st;
  int rc;
  try {
    rc = build_impl(t, pos, mass, kappa, lum, h, box_lo, box_size, st);
  } catch (const std::bad_alloc&) {
    set_error("trevr2_build: host allocation failed");
    rc = TREVR2_ENOMEM;
  }
  if (rc != TREVR2_OK) {
    std::string msg = g_err;
    free_tree(t, st);
    delete t;
    set_error("%s", msg.c_str());
    return rc;
  }
  *out = reinterpret_cast<trevr2_tree*>(t);
  return TREVR2_OK;
}

int trevr2_free(trevr2_tree* tree) {
  clear_error();
  if (!tree) return TREVR2_OK;
  Tree* t = reinterpret_cast<Tree*>(tree);
  free_tree(t, t->last_stream);
  delete t;
  return TREVR2_OK;
}

int trevr2_tree_info_get(const trevr2_tree* tree, trevr2_tree_info* info) {
  clear_error();
  if (!tree || !info) {
    set_error("trevr2_tree_info_get: NULL argument");
    return TREVR2_EINVAL;
  }
  const Tree* t = reinterpret_cast<const Tree*>(tree);
  info->n_elements = t->N;
  info->n_nodes = t->n_nodes;
  info->n_internal = t->n_internal;
  info->n_leaves = t->n_nodes - t->n_internal;
  info->nb = t->nb;
  info->bucket = t->bucket;
  info->max_depth = t->max_depth;
  info->reserved = 0;
  for (int a = 0; a < 3; ++a) info->box_lo[a] = t->lo[a];
  info->box_size = t->size;
  return TREVR2_OK;
}

}  // extern "C"

namespace trevr2 {

// Export kernels: undo the normalisation and the band padding.
__global__ void k_export_bands(const float* src, int64_t n, int nb, int nbp, float scale, float* dst) {
  int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (i >= n * nb) return;
  int64_t q = i / nb;
  int b = int(i % nb);
  dst[i] = src[q * nbp + b] * scale;
}

__global__ void k_export_centre(const double* c64, int64_t n, double lo0, double lo1, double lo2,
                                double size, double* dst) {
  int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (i >= 3 * n) return;
  double lo = (i % 3 == 0) ? lo0 : ((i % 3 == 1) ? lo1 : lo2);
  dst[i] = lo + size * c64[i];
}

__global__ void k_export_scale(const double* src, int64_t n, double scale, double* dst) {
  int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (i < n) dst[i] = src[i] * scale;
}

}  // namespace trevr2

extern "C" int trevr2_tree_export(const trevr2_tree* tree, int field, void* dst, size_t bytes,
                                  void* stream) {
  clear_error();
  if (!tree || !dst) {
    set_error("trevr2_tree_export: NULL argument");
    return TREVR2_EINVAL;
  }
  const Tree* t = reinterpret_cast<const Tree*>(tree);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int64_t N = t->N, n = t->n_nodes;
  const void* src = nullptr;
  size_t need = 0;
  switch (field) {
    case TREVR2_F_KEYS: src = t->keys; need = N * sizeof(uint64_t); break;
    case TREVR2_F_PERM: src = t->perm; need = N * sizeof(int); break;
    case TREVR2_F_PREFIX: src = t->prefix; need = n * sizeof(uint64_t); break;
    case TREVR2_F_DEPTH: src = t->depth; need = n * sizeof(int); break;
    case TREVR2_F_FIRST: src = t->first; need = n * sizeof(int); break;
    case TREVR2_F_COUNT: src = t->count; need = n * sizeof(int); break;
    case TREVR2_F_CHILD: src = t->child; need = n * sizeof(int); break;
    case TREVR2_F_PARENT: src = t->parent; need = n * sizeof(int); break;
    case TREVR2_F_LUM: need = n * t->nb * sizeof(float); break;
    case TREVR2_F_CENTRE: need = 3 * n * sizeof(double); break;
    case TREVR2_F_ALPHA_LEAF: need = n * t->nb * sizeof(float); break;
    case TREVR2_F_B: need = n * sizeof(double); break;
    default:
      set_error("trevr2_tree_export: unknown field %d", field);
      return TREVR2_EINVAL;
  }
  if (bytes < need) {
    set_error("trevr2_tree_export: destination holds %zu bytes, %zu needed", bytes, need);
    return TREVR2_EINVAL;
  }
  if (need == 0) return TREVR2_OK;
  if (src) {
    T2_CUDA(cudaMemcpyAsync(dst, src, need, cudaMemcpyDeviceToDevice, st));
  } else if (field == TREVR2_F_LUM) {
    k_export_bands<<<blocks_for(n * t->nb, 256), 256, 0, st>>>(t->Lnode, n, t->nb, t->nbp, 1.0f,
                                                                static_cast<float*>(dst)); note_launch();
  } else if (field == TREVR2_F_ALPHA_LEAF) {
    k_export_bands<<<blocks_for(n * t->nb, 256), 256, 0, st>>>(
        t->alpha_leaf, n, t->nb, t->nbp, float(1.0 / t->size), static_cast<float*>(dst)); note_launch();
  } else if (field == TREVR2_F_CENTRE) {
    k_export_centre<<<blocks_for(3 * n, 256), 256, 0, st>>>(t->c64, n, t->lo[0], t->lo[1],
                                                            t->lo[2], t->size,
                                                            static_cast<double*>(dst)); note_launch();
  } else if (field == TREVR2_F_B) {
    k_export_scale<<<blocks_for(n, 256), 256, 0, st>>>(t->B64, n, t->size,
                                                       static_cast<double*>(dst)); note_launch();
  }
  T2_CUDA(cudaGetLastError());
  return TREVR2_OK;
}

// ---------------------------------------------------------------------------
// Refinement tau_refine (Sec. 2.5.2; off by default): a cell whose optical
// depth varies by more than tau_refine inside it opens as well.  The
// variation is (largest - smallest bucket alpha among the leaves under the
// cell) times its longest side, the largest over the bands.  Opening is
// forced by a node copy whose B is so large that B > theta d holds for
// every d in the unit cube, so every walk (forward, per bucket, batched,
// adjoint) refines without any change to its code.
namespace trevr2 {

constexpr float kRefinedB = 1e18f;  // B^2 and the FP32 guard stay finite

// One depth of the tree, deepest first: the per-band range of the leaves'
// alpha under each node and the node's variation.
template <int NBP>
__global__ void k_tau_variation_level(int64_t lb, int64_t le, const NodeW* __restrict__ nodes,
                                      const float* __restrict__ alpha_leaf, float* amin,
                                      float* amax, float* __restrict__ dtau) {
  const int64_t q = lb + blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (q >= le) return;
  const NodeW nd = nodes[q];
  float var = 0.0f;
#pragma unroll
  for (int b = 0; b < NBP; ++b) {
    float lo, hi;
    if (nd.meta & kMetaLeaf) {
      lo = hi = alpha_leaf[q * NBP + b];
    } else {
      const int64_t c = nd.child;
      lo = fminf(amin[c * NBP + b], amin[(c + 1) * NBP + b]);
      hi = fmaxf(amax[c * NBP + b], amax[(c + 1) * NBP + b]);
    }
    amin[q * NBP + b] = lo;
    amax[q * NBP + b] = hi;
    var = fmaxf(var, hi - lo);
  }
  // the longest side: the axis split least often, z, floor(depth / 3) times
  const int d = int(nd.meta & kMetaDepthMask);
  dtau[q] = var * ldexpf(1.0f, -splits_on_axis(d, 2));
}

__global__ void k_refine_nodes(int64_t n, const NodeW* __restrict__ nodes,
                               const float* __restrict__ dtau, float tau,
                               NodeW* __restrict__ out) {
  const int64_t q = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (q >= n) return;
  NodeW nd = nodes[q];
  if (!(nd.meta & kMetaLeaf) && dtau[q] > tau) nd.B = kRefinedB;
  out[q] = nd;
}

}  // namespace trevr2

extern "C" int trevr2_set_tau_refine(trevr2_tree* tree, double tau_refine, void* stream) {
  clear_error();
  if (!tree) {
    set_error("trevr2_set_tau_refine: tree is NULL");
    return TREVR2_EINVAL;
  }
  if (!(tau_refine > 0.0)) {
    set_error("trevr2_set_tau_refine: tau_refine must be positive (infinity turns it off)");
    return TREVR2_EINVAL;
  }
  Tree* t = reinterpret_cast<Tree*>(tree);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (std::isinf(tau_refine)) {
    t->refine_on = false;
    t->tau_refine = tau_refine;
    return TREVR2_OK;
  }
  const int64_t n = t->n_nodes;
  if (!t->dtau) {
    // computed into temporaries and kept only when complete, so that a
    // failed call leaves the tree as it was
    DeviceTemp<float> dtau(st), range(st);
    T2_CHECK(dalloc(&dtau.p, size_t(n), st));
    T2_CHECK(dalloc(&range.p, size_t(n) * 2 * t->nbp, st));
    float* amin = range.p;
    float* amax = range.p + size_t(n) * t->nbp;
    for (int d = int(t->level_begin.size()) - 2; d >= 0; --d) {
      const int64_t lb = t->level_begin[d], le = t->level_begin[d + 1];
      if (le <= lb) continue;
      const unsigned g = blocks_for(le - lb, 256);
      switch (t->nbp) {
        case 1: k_tau_variation_level<1><<<g, 256, 0, st>>>(lb, le, t->nodes, t->alpha_leaf, amin, amax, dtau.p); break;
        case 2: k_tau_variation_level<2><<<g, 256, 0, st>>>(lb, le, t->nodes, t->alpha_leaf, amin, amax, dtau.p); break;
        default: k_tau_variation_level<4><<<g, 256, 0, st>>>(lb, le, t->nodes, t->alpha_leaf, amin, amax, dtau.p); break;
      }
      note_launch();
    }
    T2_CUDA(cudaGetLastError());
    t->dtau = dtau.p;
    dtau.p = nullptr;
  }
  if (!t->nodes_refined) T2_CHECK(dalloc(&t->nodes_refined, size_t(n), st));
  k_refine_nodes<<<blocks_for(n, 256), 256, 0, st>>>(n, t->nodes, t->dtau, float(tau_refine),
                                                      t->nodes_refined);
  note_launch();
  T2_CUDA(cudaGetLastError());
  t->refine_on = true;
  t->tau_refine = tau_refine;
  return TREVR2_OK;
}
