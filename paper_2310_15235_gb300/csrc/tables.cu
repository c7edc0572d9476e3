// Per-direction absorption tables (TREVR2, Sec. 2.6, Eq. transmissionavg).
//
// For every internal cell and every antipodal pair of HEALPix beams
// (N_ray/2 stored values per cell, Sec. 2.6), the two halves are combined by
// the volume-weighted transmission
//   T = [V1 e^{-d a1} + V2 e^{-d a2} + V12 e^{-d a1/2} e^{-d a2/2}] / V,
//   alpha = -ln(T) / d,
// with V12 the volume of points whose line along the beam crosses the shared
// face inside the cell, V1 = V2 = V/2 - V12/2, and d the chord through the
// centre of the shared face (the cell centre).  The through-ray term is the
// product of the two half-cell transmissions: the printed sum of the two
// exponentials exceeds 1 for a transparent cell and contradicts the paper's
// own worked example.  Leaves are isotropic (bucket absorption).  With
// TREVR2_LINEAR the halves are combined by their volume-weighted linear
// average instead (Sec. 2.6's comparison scheme): (alpha_1 + alpha_2) / 2,
// the same in every direction pair.
//
// Cell shapes repeat every three levels (cube split on x; 1:2:2 split on y;
// 1:1:2 split on z), so the weights depend only on (depth mod 3, beam pair)
// and the chord scales with 2^-(depth/3): they are computed once per nside in
// FP64.  The combination runs in FP32 as
//   m > 1:  ln T = -m + ln(sum_j w_j e^{-(x_j - m)})      (no underflow)
//   m <= 1: ln T = log1p(sum_j w_j expm1(-x_j)) if T > 1/2 (thin cells keep
//           their relative precision), else ln(sum_j w_j e^{-x_j}),
// where x_j are the exponents of the terms and m the smallest one with a
// nonzero weight — the same expression, evaluated stably.
#include <algorithm>

#include "healpix.cuh"
#include "internal.cuh"

namespace trevr2 {

__global__ void k_dirs(int nside, int npix, double* __restrict__ dirs64, float4* __restrict__ dirs) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= npix) return;
  double v[3];
  hp_pix2vec(nside, k, v);
  for (int a = 0; a < 3; ++a) dirs64[3 * k + a] = v[a];
  int pair = k < npix / 2 ? k : hp_vec2pix_f64(nside, -v[0], -v[1], -v[2]);
  dirs[k] = make_float4(float(v[0]), float(v[1]), float(v[2]), __int_as_float(pair));
}

// Transmission geometry of one cell shape (unit scale) for one beam pair.
__global__ void k_trans_geo(int P, const double* __restrict__ dirs64, TransGeo* __restrict__ geo) {
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= 3 * P) return;
  const int shape = idx / P, p = idx % P;
  double E[3] = {1.0, 1.0, 1.0};
  if (shape >= 1) E[0] = 0.5;
  if (shape >= 2) E[1] = 0.5;
  const int a = shape, b = (a + 1) % 3, c = (a + 2) % 3;
  const double n[3] = {dirs64[3 * p], dirs64[3 * p + 1], dirs64[3 * p + 2]};
  const double V = E[0] * E[1] * E[2];
  double V12 = 0.0;
  if (n[a] != 0.0) {
    // depth u below the shared face: the rays through points at u that reach
    // the face inside it cover (Lb - u rb)(Lc - u rc); integrate to u_max.
    const double rb = fabs(n[b] / n[a]), rc = fabs(n[c] / n[a]);
    const double Lb = E[b], Lc = E[c];
    double u = 0.5 * E[a];
    if (rb > 0.0) u = fmin(u, Lb / rb);
    if (rc > 0.0) u = fmin(u, Lc / rc);
    V12 = 2.0 * (Lb * Lc * u - 0.5 * (Lb * rc + Lc * rb) * u * u + rb * rc * u * u * u / 3.0);
  }
  double d = INFINITY;
  for (int k = 0; k < 3; ++k)
    if (n[k] != 0.0) d = fmin(d, E[k] / fabs(n[k]));
  TransGeo g;
  g.w1 = float((0.5 * V - 0.5 * V12) / V);
  g.w12 = float(V12 / V);
  g.d_unit = float(d);
  g.pad = 0.0f;
  geo[idx] = g;
}

__device__ __forceinline__ float combine_alpha(float a1, float a2, float w1, float w12, float d) {
  const float x1 = d * a1, x2 = d * a2, x12 = 0.5f * (x1 + x2);
  float m = INFINITY;
  if (w1 > 0.0f) m = fminf(x1, x2);
  if (w12 > 0.0f) m = fminf(m, x12);
  float lnT;
  if (m > 1.0f) {
    float S = 0.0f;
    if (w1 > 0.0f) S += w1 * (expf(-(x1 - m)) + expf(-(x2 - m)));
    if (w12 > 0.0f) S += w12 * expf(-(x12 - m));
    lnT = -m + logf(S);
  } else {
    float S = 0.0f;
    if (w1 > 0.0f) S += w1 * (expf(-x1) + expf(-x2));
    if (w12 > 0.0f) S += w12 * expf(-x12);
    if (S > 0.5f) {
      float e = 0.0f;
      if (w1 > 0.0f) e += w1 * (expm1f(-x1) + expm1f(-x2));
      if (w12 > 0.0f) e += w12 * expm1f(-x12);
      lnT = log1pf(e);
    } else {
      lnT = logf(S);
    }
  }
  return fmaxf(0.0f, -lnT / d);
}

template <int NBP>
__global__ void k_alpha_level(int64_t lb, int64_t le, int P, int nb, bool linear,
                              const NodeW* __restrict__ nodes,
                              const int* __restrict__ int_index,
                              const float* __restrict__ alpha_leaf,
                              const TransGeo* __restrict__ geo, float* __restrict__ tab) {
  int64_t idx = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  int64_t q = lb + idx / P;
  int p = int(idx % P);
  if (q >= le) return;
  const NodeW nd = nodes[q];
  if (nd.child < 0) return;
  const int depth = int(nd.meta & kMetaDepthMask);
  const TransGeo g = geo[(depth % 3) * P + p];
  const float d = ldexpf(g.d_unit, -(depth / 3));
  float a1[NBP], a2[NBP];
  const int c = nd.child;
  const int i1 = int_index[c], i2 = int_index[c + 1];
#pragma unroll
  for (int b = 0; b < NBP; ++b) {
    a1[b] = i1 < 0 ? alpha_leaf[int64_t(c) * NBP + b] : tab[(int64_t(i1) * P + p) * NBP + b];
    a2[b] = i2 < 0 ? alpha_leaf[int64_t(c + 1) * NBP + b] : tab[(int64_t(i2) * P + p) * NBP + b];
  }
  const int iq = int_index[q];
#pragma unroll
  for (int b = 0; b < NBP; ++b) {
    float al = 0.0f;
    if (b < nb && (a1[b] > 0.0f || a2[b] > 0.0f))
      al = linear ? 0.5f * (a1[b] + a2[b]) : combine_alpha(a1[b], a2[b], g.w1, g.w12, d);
    tab[(int64_t(iq) * P + p) * NBP + b] = al;
  }
}

int ensure_table(Tree* t, int nside, cudaStream_t st, Table** out, bool linear) {
  for (Table& tb : t->tables)
    if (tb.nside == nside && tb.linear == linear) {
      *out = &tb;
      return TREVR2_OK;
    }
  const int npix = 12 * nside * nside, P = npix / 2;
  // built in temporaries and kept by the tree only when complete
  DeviceTemp<float4> dirs(st);
  DeviceTemp<double> dirs64(st);
  DeviceTemp<TransGeo> geo(st);
  DeviceTemp<float> alpha(st);
  T2_CHECK(dalloc(&dirs.p, npix, st));
  T2_CHECK(dalloc(&dirs64.p, 3 * size_t(npix), st));
  T2_CHECK(dalloc(&geo.p, 3 * size_t(P), st));
  T2_CHECK(dalloc(&alpha.p, size_t(std::max<int64_t>(t->n_internal, 1)) * P * t->nbp, st));
  Table tb;
  tb.nside = nside;
  tb.linear = linear;
  tb.dirs = dirs.p;
  tb.dirs64 = dirs64.p;
  tb.geo = geo.p;
  tb.alpha = alpha.p;
  k_dirs<<<(npix + 127) / 128, 128, 0, st>>>(nside, npix, tb.dirs64, tb.dirs); note_launch();
  k_trans_geo<<<(3 * P + 127) / 128, 128, 0, st>>>(P, tb.dirs64, tb.geo); note_launch();
  for (int d = t->max_depth; d >= 0; --d) {
    int64_t a = t->level_begin[d], b = t->level_begin[d + 1];
    int64_t work = (b - a) * P;
    unsigned blocks = unsigned((work + 255) / 256);
    if (work == 0) continue;
    switch (t->nbp) {
      case 1: k_alpha_level<1><<<blocks, 256, 0, st>>>(a, b, P, t->nb, linear, t->nodes, t->int_index, t->alpha_leaf, tb.geo, tb.alpha); note_launch(); break;
      case 2: k_alpha_level<2><<<blocks, 256, 0, st>>>(a, b, P, t->nb, linear, t->nodes, t->int_index, t->alpha_leaf, tb.geo, tb.alpha); note_launch(); break;
      default: k_alpha_level<4><<<blocks, 256, 0, st>>>(a, b, P, t->nb, linear, t->nodes, t->int_index, t->alpha_leaf, tb.geo, tb.alpha); note_launch(); break;
    }
  }
  T2_CUDA(cudaGetLastError());
  t->tables.push_back(tb);
  dirs.p = nullptr;
  dirs64.p = nullptr;
  geo.p = nullptr;
  alpha.p = nullptr;
  *out = &t->tables.back();
  return TREVR2_OK;
}

__global__ void k_export_alpha(const NodeW* __restrict__ nodes, const int* __restrict__ int_index,
                               const float* __restrict__ alpha_leaf, const float* __restrict__ tab,
                               int64_t n, int P, int nb, int nbp, float scale, float* __restrict__ dst) {
  int64_t idx = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (idx >= n * P * nb) return;
  int64_t q = idx / (int64_t(P) * nb);
  int rem = int(idx % (int64_t(P) * nb));
  int p = rem / nb, b = rem % nb;
  int iq = int_index[q];
  float a = iq < 0 ? alpha_leaf[q * nbp + b] : tab[(int64_t(iq) * P + p) * nbp + b];
  dst[idx] = a * scale;
}

__global__ void k_pix2vec(int nside, int npix, double* __restrict__ dst) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= npix) return;
  double v[3];
  hp_pix2vec(nside, k, v);
  for (int a = 0; a < 3; ++a) dst[3 * k + a] = v[a];
}

// The walk's pixel lookup: FP32 with a guard band, FP64 when inside it.
__global__ void k_vec2pix(int nside, const double* __restrict__ v, int64_t n, int32_t* __restrict__ pix) {
  int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (i >= n) return;
  double x = v[3 * i], y = v[3 * i + 1], z = v[3 * i + 2];
  float fx = float(x), fy = float(y), fz = float(z);
  float r = sqrtf(fx * fx + fy * fy + fz * fz);
  int p = hp_vec2pix_f32(nside, fx, fy, fz, hp_guard(nside, r));
  if (p < 0) p = hp_vec2pix_f64(nside, x, y, z);
  pix[i] = p;
}

static bool valid_nside(int nside) {
  return nside >= 1 && nside <= TREVR2_MAX_NSIDE && (nside & (nside - 1)) == 0;
}

}  // namespace trevr2

using namespace trevr2;

extern "C" int trevr2_alpha_table(trevr2_tree* tree, int nside, float* dst, size_t bytes,
                                  void* stream) {
  clear_error();
  if (!tree || !dst) {
    set_error("trevr2_alpha_table: NULL argument");
    return TREVR2_EINVAL;
  }
  if (!valid_nside(nside)) {
    set_error("trevr2_alpha_table: nside %d is not a power of two in [1, %d]", nside, TREVR2_MAX_NSIDE);
    return TREVR2_EINVAL;
  }
  Tree* t = reinterpret_cast<Tree*>(tree);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  t->last_stream = st;
  const int P = 6 * nside * nside;
  const size_t need = size_t(t->n_nodes) * P * t->nb * sizeof(float);
  if (bytes < need) {
    set_error("trevr2_alpha_table: destination holds %zu bytes, %zu needed", bytes, need);
    return TREVR2_EINVAL;
  }
  Table* tb = nullptr;
  T2_CHECK(ensure_table(t, nside, st, &tb));
  int64_t total = t->n_nodes * int64_t(P) * t->nb;
  if (total > 0)
    k_export_alpha<<<unsigned((total + 255) / 256), 256, 0, st>>>(
        t->nodes, t->int_index, t->alpha_leaf, tb->alpha, t->n_nodes, P, t->nb, t->nbp,
        float(1.0 / t->size), dst); note_launch();
  T2_CUDA(cudaGetLastError());
  return TREVR2_OK;
}

extern "C" int trevr2_healpix_pix2vec(int nside, double* dst, void* stream) {
  clear_error();
  if (!dst || !valid_nside(nside)) {
    set_error("trevr2_healpix_pix2vec: NULL destination or bad nside %d", nside);
    return TREVR2_EINVAL;
  }
  int npix = 12 * nside * nside;
  k_pix2vec<<<(npix + 127) / 128, 128, 0, static_cast<cudaStream_t>(stream)>>>(nside, npix, dst); note_launch();
  T2_CUDA(cudaGetLastError());
  return TREVR2_OK;
}

extern "C" int trevr2_healpix_vec2pix(int nside, const double* v, int64_t n, int32_t* pix, void* stream) {
  clear_error();
  if (n < 0 || (n > 0 && (!v || !pix)) || !valid_nside(nside)) {
    set_error("trevr2_healpix_vec2pix: bad arguments (nside %d, n %lld)", nside, (long long)n);
    return TREVR2_EINVAL;
  }
  if (n > 0)
    k_vec2pix<<<unsigned((n + 255) / 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(nside, v, n, pix); note_launch();
  T2_CUDA(cudaGetLastError());
  return TREVR2_OK;
}
