// TREVR2 reverse ray trace: plain, slow FP64 CPU oracle.
//
// TEST INFRASTRUCTURE ONLY.  This file restates, step by step, what the
// TREVR2 method (Wadsley, Baumschlager & Shen, arXiv:2310.15235) computes for
// one radiation step: the radiation tree (Sec. 2.3), bucket absorption
// (Sec. 2.6, bucket formula), the transmission average (Eq. transmissionavg),
// HEALPix beams (Sec. 1.3, Sec. 2.5), the cell opening criterion B/d > theta
// (Sec. 2.5.2), the per-beam optical depth with the projected-distance
// correction (Sec. 2.5.1), and the optional finite-size (Eq. intint) and
// optically-thick (Eq. taucorr) factors; with flags, the per-bucket walk
// (Sec. 2.5), particle-particle absorption (Sec. 2.4), the complex source
// model (Sec. 2.7), linear averaging (Sec. 2.6), directed rays (Sec. 3.4.1)
// and absorption refinement (Sec. 2.5.2).  Only the tests, the smoke check and
// the CPU baseline of the benchmark may load it; the product library never
// does, and the two share no code, headers or tables.
//
// Plain means: no blocking, no fusion, no queues, no reordering beyond what
// the definitions state.  Every sum is a plain loop in FP64.  The method's
// discrete choices (cut, beam of each source) are taken on FP64 values.
//
// Readings of the paper that this file fixes (each is also listed in the
// design notes):
//  R1 Tree: splitting each cell at the middle of its longest side, from a
//     cube root, is cyclic x,y,z bisection (ties x<y<z), i.e. the bisection of 63-bit Morton keys
//     (21 bits per axis, bit 62 = x MSB).  Cells are the geometric bisection
//     boxes, not tight particle bounds.  A node splits iff it holds more than
//     `bucket` elements and depth < 63; empty halves are empty leaves.
//  R2 One band-summed centre of luminosity per cell (band-independent
//     geometry); the box centre if the cell has no luminosity.
//  R3 Bucket absorption alpha = sum(kappa*m) / V_box (the paper's
//     sum(kappa m)/sum(m/rho) with the box volume standing in for sum(m/rho),
//     which the inputs do not carry).
//  R4 Eq. transmissionavg: the through-ray term is the product
//     V12 exp(-d a1/2) exp(-d a2/2); the printed sum of the two exponentials
//     gives T > 1 at alpha = 0 and contradicts the paper's own worked example.
//     V12 is the volume of points whose line along the beam crosses the
//     shared face inside the box; d is the chord through the face centre.
//  R5 Absorption along a beam uses the cut: accepted cells (an internal cell
//     with its per-direction alpha, a leaf with its isotropic alpha) and
//     opened leaves (isotropic alpha), i.e. volumetric absorption also next
//     to the receiver.  The receiver never counts itself as a source.
//  R6 J is the integrated intensity (integral of I over solid angle); its
//     far-field kernel is L/(4 pi r^2).
//  R7 Finite-size kernel radius (3/(4 pi))^(1/2) h = 0.48860 h.
//  R8 Graze tie-break: boxes are half-open [lo, hi) on each axis.
//  R9 FLAG_LINEAR replaces Eq. transmissionavg by the volume-weighted linear
//     average of the two halves' absorption, the scheme Sec. 2.6 compares
//     it with; it is direction independent (the same value in every pair).
//  R10 FLAG_BUCKET (per-bucket beams, Sec. 2 and Sec. 2.5.1): the walk starts
//     from the centre of the receiver's bucket (the geometric centre of its
//     leaf box), so every receiver of a bucket shares the cut, the beam of
//     each source and the projected distance s.  Per receiver, the optical
//     depth up to s is multiplied by r/s with r the receiver's own distance
//     to the source, and the kernel is g(r).  A source at the bucket centre
//     itself has no beam and is skipped, as one on top of a receiver is.
//  R11 FLAG_PP (with FLAG_BUCKET; Sec. 2.4, Sec. 2.5): the p-p radius r_pp of
//     a bucket starts at the radius of the sphere through its box corners and
//     grows to h_j / sqrt(4 pi / N_ray) for the largest gas element j (m > 0)
//     within r_pp of the bucket centre, until no element inside is larger
//     than the beam width r_pp sqrt(4 pi / N_ray) there.  Those elements are
//     the bucket's p-p particles.  Cells whose box comes within r_pp of the
//     centre open (sources there are single elements), beams count cell
//     absorption only beyond r_pp, and per receiver and source every p-p
//     particle j (not the receiver, not the source) that is closer to the
//     source than the receiver is and lies within h_j of the receiver-source
//     segment (distance b) adds kappa_j Sigma_j(b), Sigma_j(b) =
//     3 m_j / (pi h_j^2) (1 - b / h_j), whose area integral over b < h_j is m_j.
//  R12 Directed rays (with FLAG_BUCKET; Sec. 3.4.1): given a target point,
//     the beam that holds the target's direction from the bucket centre is
//     aimed at the target instead of along its pixel centre; it keeps its
//     pixel's direction pair for the cells' absorption, and the sources
//     binned into it take their projected distance along the new direction.
//     A target at the bucket centre leaves every beam as it is.
//  R13 Refinement tau_refine (Sec. 2.5.2; off, i.e. infinite, by default):
//     a cell whose optical depth varies by more than tau_refine inside it
//     also opens.  The variation is read as (largest - smallest bucket alpha
//     among the leaves under the cell) times the cell's longest side, the
//     largest over the bands.  Leaves are buckets and never open further.
//  R14 Complex source model (FLAG_CSM, with FLAG_BUCKET; Sec. 2.7, Eq.
//     srccomb): every luminous cell keeps, per HEALPix direction k, the
//     length d_k from its centre of luminosity to its box edge along n_k and
//     the optical depth tau_k of that ray.  A leaf's is its bucket alpha
//     times d_k.  A parent's ray ends on the plane through the end of its
//     own ray, perpendicular to n_k; each luminous child's ray is clipped to
//     that plane (alpha_child times the shorter length) or extended to it,
//     the extension absorbing with the sibling's alpha (its direction pair)
//     over its chord with the sibling's box; L e^{-tau} = sum over children
//     of L_i e^{-tau_i'} per band.  In the walk, an accepted cell's source
//     takes the beam's absorption only up to its projected edge s - d_k',
//     k' the direction from the source back towards the bucket (the pixel of
//     -n_k), and adds its own tau_k'; single-element sources are as before.

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <limits>
#include <memory>
#include <thread>
#include <vector>

namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr int kKeyBitsPerAxis = 21;
constexpr int kMaxDepth = 63;

// ---------------------------------------------------------------------------
// Forward-mode dual number, used to differentiate the oracle with respect to
// one chosen input (a kappa or a luminosity).  Discrete choices always look
// at the value part, so the dual pass follows the same cut and beams.
struct Dual {
  double v = 0.0;
  double d = 0.0;
  Dual() = default;
  Dual(double value) : v(value), d(0.0) {}  // NOLINT: implicit by design
  Dual(double value, double deriv) : v(value), d(deriv) {}
};
inline Dual operator+(Dual a, Dual b) { return {a.v + b.v, a.d + b.d}; }
inline Dual operator-(Dual a, Dual b) { return {a.v - b.v, a.d - b.d}; }
inline Dual operator-(Dual a) { return {-a.v, -a.d}; }
inline Dual operator*(Dual a, Dual b) { return {a.v * b.v, a.d * b.v + a.v * b.d}; }
inline Dual operator/(Dual a, Dual b) {
  return {a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v)};
}
inline Dual& operator+=(Dual& a, Dual b) { a = a + b; return a; }
inline Dual& operator*=(Dual& a, Dual b) { a = a * b; return a; }
inline Dual exp(Dual a) { double e = std::exp(a.v); return {e, a.d * e}; }
inline Dual log(Dual a) { return {std::log(a.v), a.d / a.v}; }
inline Dual sqrt(Dual a) { double s = std::sqrt(a.v); return {s, s > 0 ? a.d / (2.0 * s) : 0.0}; }
inline Dual expm1(Dual a) { return {std::expm1(a.v), a.d * std::exp(a.v)}; }
inline double val(double x) { return x; }
inline double val(const Dual& x) { return x.v; }
using std::exp;
using std::expm1;
using std::log;
using std::sqrt;

// ---------------------------------------------------------------------------
// Sec. 2.3 / R1: Morton keys.
uint64_t morton_key(const double x[3], const double lo[3], double size) {
  uint64_t k[3];
  for (int a = 0; a < 3; ++a) {
    double u = (x[a] - lo[a]) / size;
    double f = std::floor(u * 2097152.0);  // 2^21
    if (f < 0.0) f = 0.0;
    if (f > 2097151.0) f = 2097151.0;
    k[a] = static_cast<uint64_t>(f);
  }
  uint64_t key = 0;
  for (int level = 0; level < kKeyBitsPerAxis; ++level) {
    for (int a = 0; a < 3; ++a) {
      uint64_t bit = (k[a] >> (kKeyBitsPerAxis - 1 - level)) & 1u;
      key = (key << 1) | bit;
    }
  }
  return key;
}

struct Node {
  uint64_t prefix = 0;  // key bits above the node's depth, lower bits zero
  int depth = 0;
  int64_t first = 0;    // first element (sorted order)
  int64_t count = 0;
  int64_t child = -1;   // index of the lower child; the upper child is child+1
  int64_t parent = -1;
};

// Geometric box of a node in physical coordinates (R1).
void node_box(const Node& nd, const double lo[3], double size, double blo[3], double bhi[3]) {
  double l[3] = {0.0, 0.0, 0.0};
  double e[3] = {1.0, 1.0, 1.0};
  for (int level = 0; level < nd.depth; ++level) {
    int a = level % 3;
    e[a] *= 0.5;
    if ((nd.prefix >> (kMaxDepth - 1 - level)) & 1u) l[a] += e[a];
  }
  for (int a = 0; a < 3; ++a) {
    blo[a] = lo[a] + size * l[a];
    bhi[a] = lo[a] + size * (l[a] + e[a]);
  }
}

// ---------------------------------------------------------------------------
// HEALPix, RING scheme (Gorski et al. 2005), written from its formulas:
// ring i (1..4n-1) from the north pole; polar rings hold 4i pixels at
// z = 1 - i^2/(3n^2) and phi = pi/(2i) (j + 1/2); equatorial rings
// (n <= i <= 3n) hold 4n pixels at z = (4n - 2i)/(3n) and
// phi = pi/(2n) (j + s/2) with s = 1 on rings n, n+2, ...; south mirrors north.
void pix2vec_ring(int nside, int64_t p, double v[3]) {
  const int64_t n = nside;
  const int64_t npix = 12 * n * n;
  const int64_t ncap = 2 * n * (n - 1);
  double z, phi;
  if (p < ncap) {
    int64_t i = 1;
    while (2 * i * (i + 1) <= p) ++i;
    int64_t j = p - 2 * i * (i - 1);
    z = 1.0 - static_cast<double>(i * i) / (3.0 * static_cast<double>(n * n));
    phi = kPi / (2.0 * static_cast<double>(i)) * (static_cast<double>(j) + 0.5);
  } else if (p < npix - ncap) {
    int64_t q = p - ncap;
    int64_t ir = q / (4 * n) + 1;  // 1 .. 2n+1
    int64_t j = q % (4 * n);
    int64_t i = n + ir - 1;
    z = 2.0 * static_cast<double>(2 * n - i) / (3.0 * static_cast<double>(n));
    double shift = (ir % 2 == 1) ? 0.5 : 0.0;
    phi = kPi / (2.0 * static_cast<double>(n)) * (static_cast<double>(j) + shift);
  } else {
    int64_t q = npix - 1 - p;
    int64_t i = 1;
    while (2 * i * (i + 1) <= q) ++i;
    int64_t ring_start = npix - 2 * i * (i + 1);
    int64_t j = p - ring_start;
    z = -(1.0 - static_cast<double>(i * i) / (3.0 * static_cast<double>(n * n)));
    phi = kPi / (2.0 * static_cast<double>(i)) * (static_cast<double>(j) + 0.5);
  }
  double st = std::sqrt((1.0 - z) * (1.0 + z));
  v[0] = st * std::cos(phi);
  v[1] = st * std::sin(phi);
  v[2] = z;
  // Exact zeros of the ideal centre (phi a multiple of pi/2) are lost to the
  // rounding of pi; restore them so beams in a coordinate plane stay in it.
  for (int a = 0; a < 3; ++a)
    if (std::fabs(v[a]) < 1e-15) v[a] = 0.0;
}

int64_t vec2pix_ring(int nside, const double v[3]) {
  const int64_t n = nside;
  const int64_t npix = 12 * n * n;
  const int64_t ncap = 2 * n * (n - 1);
  double norm = std::sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
  double z = v[2] / norm;
  double phi = std::atan2(v[1], v[0]);
  if (phi < 0.0) phi += 2.0 * kPi;
  double za = std::fabs(z);
  double tt = phi / (0.5 * kPi);  // in [0, 4]
  if (za <= 2.0 / 3.0) {
    double t1 = static_cast<double>(n) * (0.5 + tt);
    double t2 = static_cast<double>(n) * z * 0.75;
    int64_t jp = static_cast<int64_t>(std::floor(t1 - t2));  // ascending edge index
    int64_t jm = static_cast<int64_t>(std::floor(t1 + t2));  // descending edge index
    int64_t ir = n + 1 + jp - jm;                            // 1 .. 2n+1
    int64_t kshift = 1 - (ir & 1);
    int64_t ip = (jp + jm - n + kshift + 1) / 2;
    ip = ((ip % (4 * n)) + 4 * n) % (4 * n);
    return ncap + (ir - 1) * 4 * n + ip;
  }
  double tp = tt - std::floor(tt);
  double tmp = static_cast<double>(n) * std::sqrt(3.0 * (1.0 - za));
  int64_t jp = static_cast<int64_t>(std::floor(tp * tmp));
  int64_t jm = static_cast<int64_t>(std::floor((1.0 - tp) * tmp));
  int64_t ir = jp + jm + 1;  // ring counted from the nearer pole
  int64_t ip = static_cast<int64_t>(std::floor(tt * static_cast<double>(ir)));
  ip = ((ip % (4 * ir)) + 4 * ir) % (4 * ir);
  if (z > 0.0) return 2 * ir * (ir - 1) + ip;
  return npix - 2 * ir * (ir + 1) + ip;
}

// Each pair of antipodal beams shares one stored alpha (Sec. 2.6: N_ray/2
// values per cell).  Pair index of pixel k: k itself in the northern half of
// the RING order, else the index of its antipode.
int64_t pair_of_pixel(int nside, int64_t k) {
  int64_t npix = 12 * static_cast<int64_t>(nside) * nside;
  if (k < npix / 2) return k;
  double v[3];
  pix2vec_ring(nside, k, v);
  double w[3] = {-v[0], -v[1], -v[2]};
  return vec2pix_ring(nside, w);
}

// ---------------------------------------------------------------------------
// Eq. transmissionavg (R4).  Parent box extents E, split axis a, beam
// direction n.  Returns weights V1/V, V2/V, V12/V and the chord d.
struct TransGeo {
  double w1, w2, w12, d, V1, V2, V12, V;
};

TransGeo transmission_geometry(const double E[3], int a, const double n[3]) {
  int b = (a + 1) % 3, c = (a + 2) % 3;
  double w = 0.5 * E[a];  // half width along the split axis
  double Lb = E[b], Lc = E[c];
  double V = E[0] * E[1] * E[2];
  double V12 = 0.0;
  if (n[a] != 0.0) {
    // Points at depth u from the shared face whose line along n reaches the
    // face inside it: (Lb - u rb)(Lc - u rc) per unit depth, both halves.
    double rb = std::fabs(n[b] / n[a]);
    double rc = std::fabs(n[c] / n[a]);
    double umax = w;
    if (rb > 0.0) umax = std::min(umax, Lb / rb);
    if (rc > 0.0) umax = std::min(umax, Lc / rc);
    double u = umax;
    double one_half = Lb * Lc * u - 0.5 * (Lb * rc + Lc * rb) * u * u + rb * rc * u * u * u / 3.0;
    V12 = 2.0 * one_half;
  }
  double VH = 0.5 * V;
  double V1 = VH - 0.5 * V12;
  double V2 = VH - 0.5 * V12;
  // Chord through the face centre (= the parent box centre) along n.
  double d = std::numeric_limits<double>::infinity();
  for (int k = 0; k < 3; ++k)
    if (n[k] != 0.0) d = std::min(d, E[k] / std::fabs(n[k]));
  TransGeo g;
  g.V1 = V1; g.V2 = V2; g.V12 = V12; g.V = V;
  g.w1 = V1 / V; g.w2 = V2 / V; g.w12 = V12 / V; g.d = d;
  return g;
}

template <class T>
T transmission_alpha(const T& a1, const T& a2, const TransGeo& g) {
  // T = [V1 e^{-d a1} + V2 e^{-d a2} + V12 e^{-d a1/2} e^{-d a2/2}] / V and
  // alpha = -ln(T)/d.  The smallest exponent is factored out of the sum so
  // that thick cells do not underflow; this is the same expression.
  T x1 = g.d * a1;
  T x2 = g.d * a2;
  T x12 = 0.5 * (x1 + x2);
  double m = std::numeric_limits<double>::infinity();
  if (g.w1 > 0.0) m = std::min(m, val(x1));
  if (g.w2 > 0.0) m = std::min(m, val(x2));
  if (g.w12 > 0.0) m = std::min(m, val(x12));
  T S = 0.0;
  if (g.w1 > 0.0) S += g.w1 * exp(-(x1 - m));
  if (g.w2 > 0.0) S += g.w2 * exp(-(x2 - m));
  if (g.w12 > 0.0) S += g.w12 * exp(-(x12 - m));
  T alpha = (T(m) - log(S)) / g.d;
  if (val(alpha) < 0.0) alpha = T(0.0);  // T >= 1 only by rounding
  return alpha;
}

// ---------------------------------------------------------------------------
// Eq. intint (finite-size element, R7) as a kernel g(r) = <4 pi J>/L, and
// Eq. taucorr (optically thick element).
constexpr double kSoftRadius = 0.48860251190291992;  // sqrt(3/(4 pi))

template <class T>
T soft_kernel(const T& r, double h) {
  T x = r / (kSoftRadius * h);
  double xv = val(x);
  T g;
  if (xv == 0.0) {
    g = T(1.0);  // limit of the closed form at x -> 0 (peak 1/h^2)
  } else if (xv == 1.0) {
    g = T(0.5);  // removable point: (x^2-1) ln((x-1)^2) -> 0
  } else if (xv <= 2.0) {
    T ratio = ((x - 1.0) * (x - 1.0)) / ((x + 1.0) * (x + 1.0));
    g = 0.5 * (T(1.0) + (x * x - 1.0) / (4.0 * x) * log(ratio));
  } else {
    // The same function through the expansion of the logarithm:
    // 1 + (x^2-1)/(4x) ln((x-1)^2/(x+1)^2) = sum_{m>=1} 2 x^{-2m}/(4m^2-1),
    // which avoids the cancellation of the closed form at large x.
    T ix2 = T(1.0) / (x * x);
    T xm = T(1.0);
    T s = T(0.0);
    for (int m = 1; m < 400; ++m) {
      xm = xm * ix2;
      T term = xm / (4.0 * m * m - 1.0);
      s += term;
      if (val(term) < 1e-18 * val(s)) break;
    }
    g = s;
  }
  return g / (h * h);
}

template <class T>
T thick_factor(const T& tau) {
  if (val(tau) == 0.0) return T(1.0);
  return -expm1(-tau) / tau;
}

// ---------------------------------------------------------------------------
struct Tree {
  int64_t N = 0;
  int nb = 0;
  int bucket = 12;
  double lo[3] = {0, 0, 0};
  double size = 1.0;
  std::vector<double> pos;    // [N][3] original order
  std::vector<double> mass;   // [N]
  std::vector<double> kappa;  // [N][nb]
  std::vector<double> lum;    // [N][nb]
  std::vector<double> h;      // [N] element size used by SOFT and THICK
  std::vector<uint64_t> key;  // [N] original order
  std::vector<int64_t> perm;  // sorted position -> original index
  std::vector<Node> nodes;    // breadth first, by prefix within a depth
  int max_depth = 0;
};

template <class T>
struct Aggregates {
  std::vector<T> L;       // [n][nb] summed luminosity
  std::vector<T> Ltot;    // [n]
  std::vector<T> c;       // [n][3] centre of luminosity
  std::vector<T> alpha;   // [n][nb] bucket absorption (leaves; 0 for internal)
  std::vector<double> B;  // [n] max distance from c to a box corner
};

// Sec. 2.5.2: B is the largest distance from the centre of luminosity to
// the cell edge, i.e. to the farthest of the 8 box corners.
double max_corner_distance(const double c[3], const double blo[3], const double bhi[3]) {
  double B2 = 0.0;
  for (int corner = 0; corner < 8; ++corner) {
    double r2 = 0.0;
    for (int a = 0; a < 3; ++a) {
      double p = ((corner >> a) & 1) ? bhi[a] : blo[a];
      double dd = p - c[a];
      r2 += dd * dd;
    }
    B2 = std::max(B2, r2);
  }
  return std::sqrt(B2);
}

// Distance from a point to the closed box (0 inside or on it).
double box_distance(const double x[3], const double blo[3], const double bhi[3]) {
  double s = 0.0;
  for (int a = 0; a < 3; ++a) {
    double dd = 0.0;
    if (x[a] < blo[a]) dd = blo[a] - x[a];
    else if (x[a] > bhi[a]) dd = x[a] - bhi[a];
    s += dd * dd;
  }
  return std::sqrt(s);
}

// Sec. 2.5.2 opening criterion: open iff d == 0 (a cell always opens itself)
// or B > theta d, d being the distance to the closest point of the cell.
bool cell_opens(const double x[3], const double blo[3], const double bhi[3], double B,
                double theta) {
  double d = box_distance(x, blo, bhi);
  return (d == 0.0) || (B > theta * d);
}

void build_tree(Tree& t) {
  const int64_t N = t.N;
  t.key.resize(N);
  for (int64_t i = 0; i < N; ++i) t.key[i] = morton_key(&t.pos[3 * i], t.lo, t.size);
  t.perm.resize(N);
  for (int64_t i = 0; i < N; ++i) t.perm[i] = i;
  std::stable_sort(t.perm.begin(), t.perm.end(),
                   [&](int64_t a, int64_t b) { return t.key[a] < t.key[b]; });
  t.nodes.clear();
  Node root;
  root.first = 0;
  root.count = N;
  t.nodes.push_back(root);
  t.max_depth = 0;
  for (size_t q = 0; q < t.nodes.size(); ++q) {
    Node nd = t.nodes[q];
    t.max_depth = std::max(t.max_depth, nd.depth);
    if (!(nd.count > t.bucket && nd.depth < kMaxDepth)) continue;
    int bit = kMaxDepth - 1 - nd.depth;
    int64_t m = nd.first;
    while (m < nd.first + nd.count && ((t.key[t.perm[m]] >> bit) & 1u) == 0) ++m;
    Node lo_child, hi_child;
    lo_child.prefix = nd.prefix;
    hi_child.prefix = nd.prefix | (uint64_t(1) << bit);
    lo_child.depth = hi_child.depth = nd.depth + 1;
    lo_child.first = nd.first;
    lo_child.count = m - nd.first;
    hi_child.first = m;
    hi_child.count = nd.first + nd.count - m;
    lo_child.parent = hi_child.parent = static_cast<int64_t>(q);
    t.nodes[q].child = static_cast<int64_t>(t.nodes.size());
    t.nodes.push_back(lo_child);
    t.nodes.push_back(hi_child);
  }
}

// L_b, centre of luminosity (R2), bucket absorption (R3) and B (Sec. 2.5.2).
// Each node's sums run over its own elements in sorted order.
template <class T>
Aggregates<T> compute_aggregates(const Tree& t, const std::vector<T>& kappa,
                                 const std::vector<T>& lum) {
  const int64_t n = static_cast<int64_t>(t.nodes.size());
  const int nb = t.nb;
  Aggregates<T> ag;
  ag.L.assign(n * nb, T(0.0));
  ag.Ltot.assign(n, T(0.0));
  ag.c.assign(n * 3, T(0.0));
  ag.alpha.assign(n * nb, T(0.0));
  ag.B.assign(n, 0.0);
  for (int64_t q = 0; q < n; ++q) {
    const Node& nd = t.nodes[q];
    double blo[3], bhi[3];
    node_box(nd, t.lo, t.size, blo, bhi);
    T Lt = 0.0;
    T cs[3] = {0.0, 0.0, 0.0};
    for (int64_t e = nd.first; e < nd.first + nd.count; ++e) {
      int64_t i = t.perm[e];
      T li = 0.0;
      for (int b = 0; b < nb; ++b) {
        ag.L[q * nb + b] += lum[i * nb + b];
        li += lum[i * nb + b];
      }
      Lt += li;
      for (int a = 0; a < 3; ++a) cs[a] += li * t.pos[3 * i + a];
    }
    ag.Ltot[q] = Lt;
    for (int a = 0; a < 3; ++a)
      ag.c[3 * q + a] = (val(Lt) > 0.0) ? cs[a] / Lt : T(0.5 * (blo[a] + bhi[a]));
    double cv[3] = {val(ag.c[3 * q]), val(ag.c[3 * q + 1]), val(ag.c[3 * q + 2])};
    ag.B[q] = max_corner_distance(cv, blo, bhi);
    if (nd.child < 0) {
      double V = (bhi[0] - blo[0]) * (bhi[1] - blo[1]) * (bhi[2] - blo[2]);
      for (int b = 0; b < nb; ++b) {
        T s = 0.0;
        for (int64_t e = nd.first; e < nd.first + nd.count; ++e) {
          int64_t i = t.perm[e];
          s += kappa[i * nb + b] * t.mass[i];
        }
        ag.alpha[q * nb + b] = s / V;
      }
    }
  }
  return ag;
}

// Per-direction-pair alpha for every node: leaves repeat their isotropic
// alpha; internal nodes combine their two halves by Eq. transmissionavg, or
// (linear) by the volume-weighted linear average of the halves' absorption
// that Sec. 2.6 compares it with, deepest nodes first so children are done
// before parents.
template <class T>
std::vector<T> alpha_tables(const Tree& t, const Aggregates<T>& ag, int nside, bool linear) {
  const int64_t n = static_cast<int64_t>(t.nodes.size());
  const int nb = t.nb;
  const int64_t P = 6 * static_cast<int64_t>(nside) * nside;
  std::vector<T> tab(n * P * nb, T(0.0));
  std::vector<double> dirs(P * 3);
  for (int64_t p = 0; p < P; ++p) pix2vec_ring(nside, p, &dirs[3 * p]);
  for (int64_t q = n - 1; q >= 0; --q) {
    const Node& nd = t.nodes[q];
    if (nd.child < 0) {
      for (int64_t p = 0; p < P; ++p)
        for (int b = 0; b < nb; ++b) tab[(q * P + p) * nb + b] = ag.alpha[q * nb + b];
      continue;
    }
    double blo[3], bhi[3];
    node_box(nd, t.lo, t.size, blo, bhi);
    double E[3] = {bhi[0] - blo[0], bhi[1] - blo[1], bhi[2] - blo[2]};
    int axis = nd.depth % 3;
    int64_t c1 = nd.child, c2 = nd.child + 1;
    if (linear) {
      // alpha = (V_1 alpha_1 + V_2 alpha_2) / V over the two halves' boxes
      double lo1[3], hi1[3], lo2[3], hi2[3];
      node_box(t.nodes[c1], t.lo, t.size, lo1, hi1);
      node_box(t.nodes[c2], t.lo, t.size, lo2, hi2);
      const double V = E[0] * E[1] * E[2];
      const double V1 = (hi1[0] - lo1[0]) * (hi1[1] - lo1[1]) * (hi1[2] - lo1[2]);
      const double V2 = (hi2[0] - lo2[0]) * (hi2[1] - lo2[1]) * (hi2[2] - lo2[2]);
      for (int64_t p = 0; p < P; ++p)
        for (int b = 0; b < nb; ++b)
          tab[(q * P + p) * nb + b] =
              (V1 * tab[(c1 * P + p) * nb + b] + V2 * tab[(c2 * P + p) * nb + b]) / V;
      continue;
    }
    for (int64_t p = 0; p < P; ++p) {
      TransGeo g = transmission_geometry(E, axis, &dirs[3 * p]);
      for (int b = 0; b < nb; ++b) {
        T a1 = tab[(c1 * P + p) * nb + b];
        T a2 = tab[(c2 * P + p) * nb + b];
        tab[(q * P + p) * nb + b] = transmission_alpha(a1, a2, g);
      }
    }
  }
  return tab;
}

// Chord [t0, t1] of the ray x + t n (t >= 0) with the half-open box (R8).
bool ray_chord(const double x[3], const double n[3], const double blo[3], const double bhi[3],
               double& t0, double& t1) {
  t0 = 0.0;
  t1 = std::numeric_limits<double>::infinity();
  for (int a = 0; a < 3; ++a) {
    if (n[a] == 0.0) {
      if (!(blo[a] <= x[a] && x[a] < bhi[a])) return false;
      continue;
    }
    double ta = (blo[a] - x[a]) / n[a];
    double tb = (bhi[a] - x[a]) / n[a];
    if (ta > tb) std::swap(ta, tb);
    t0 = std::max(t0, ta);
    t1 = std::min(t1, tb);
  }
  return t1 > t0;
}

template <class F>
void parallel_for(int64_t n, int nthreads, F&& f) {
  if (nthreads <= 0) nthreads = static_cast<int>(std::max(1u, std::thread::hardware_concurrency()));
  if (nthreads == 1 || n < 2) {
    for (int64_t i = 0; i < n; ++i) f(i);
    return;
  }
  std::atomic<int64_t> next(0);
  std::vector<std::thread> pool;
  for (int w = 0; w < nthreads; ++w)
    pool.emplace_back([&]() {
      for (;;) {
        int64_t i = next.fetch_add(1);
        if (i >= n) break;
        f(i);
      }
    });
  for (auto& th : pool) th.join();
}

enum : uint32_t { FLAG_SOFT = 1u, FLAG_THICK = 2u, FLAG_LINEAR = 8u, FLAG_BUCKET = 16u,
                  FLAG_PP = 32u, FLAG_CSM = 64u };

// R14: the complex source model's per-cell, per-direction rays.
struct CsmTables {
  std::vector<double> d;    // [n][npix] length from the centre of luminosity to the edge
  std::vector<double> tau;  // [n][npix][nb]
  std::vector<int64_t> anti;  // [npix] pixel of -n_k
};

CsmTables csm_tables(const Tree& t, const Aggregates<double>& ag, const std::vector<double>& tab,
                     int nside) {
  const int64_t n = static_cast<int64_t>(t.nodes.size());
  const int nb = t.nb;
  const int64_t npix = 12 * static_cast<int64_t>(nside) * nside;
  const int64_t P = npix / 2;
  std::vector<double> dirs(npix * 3);
  CsmTables cs;
  cs.anti.resize(npix);
  for (int64_t k = 0; k < npix; ++k) pix2vec_ring(nside, k, &dirs[3 * k]);
  for (int64_t k = 0; k < npix; ++k) {
    double m[3] = {-dirs[3 * k], -dirs[3 * k + 1], -dirs[3 * k + 2]};
    cs.anti[k] = vec2pix_ring(nside, m);
  }
  cs.d.assign(n * npix, 0.0);
  cs.tau.assign(n * npix * nb, 0.0);
  // directions are independent: one worker per direction, cells from the
  // leaves up (children come after their parent in breadth-first order)
  parallel_for(npix, 0, [&](int64_t k) {
   const double* nk = &dirs[3 * k];
   for (int64_t q = n - 1; q >= 0; --q) {
    if (!(ag.Ltot[q] > 0.0)) continue;
    const Node& nd = t.nodes[q];
    double lo[3], hi[3];
    node_box(nd, t.lo, t.size, lo, hi);
    const double* c = &ag.c[3 * q];
    {
      double t0, t1;
      const double d = ray_chord(c, nk, lo, hi, t0, t1) ? t1 : 0.0;
      cs.d[q * npix + k] = d;
      double* tq = &cs.tau[(q * npix + k) * nb];
      if (nd.child < 0) {
        for (int b = 0; b < nb; ++b) tq[b] = ag.alpha[q * nb + b] * d;
        continue;
      }
      std::vector<double> sum(nb, 0.0);
      for (int64_t i = nd.child; i <= nd.child + 1; ++i) {
        if (!(ag.Ltot[i] > 0.0)) continue;
        const int64_t sib = (i == nd.child) ? nd.child + 1 : nd.child;
        const double* ci = &ag.c[3 * i];
        // the child's ray to the parent's end plane
        double D = d;
        for (int a = 0; a < 3; ++a) D += (c[a] - ci[a]) * nk[a];
        D = std::max(D, 0.0);
        const double di = cs.d[i * npix + k];
        double ext = 0.0;  // the extension's chord with the sibling's box
        if (D > di) {
          double slo[3], shi[3], s0, s1;
          node_box(t.nodes[sib], t.lo, t.size, slo, shi);
          if (ray_chord(ci, nk, slo, shi, s0, s1))
            ext = std::max(0.0, std::min(s1, D) - std::max(s0, di));
        }
        for (int b = 0; b < nb; ++b) {
          const double ti = cs.tau[(i * npix + k) * nb + b];
          double tc;
          if (D <= di) tc = di > 0.0 ? ti * (D / di) : 0.0;
          else tc = ti + tab[(sib * P + pair_of_pixel(nside, k)) * nb + b] * ext;
          sum[b] += ag.L[i * nb + b] * std::exp(-tc);
        }
      }
      for (int b = 0; b < nb; ++b)
        tq[b] = ag.L[q * nb + b] > 0.0 ? -std::log(sum[b] / ag.L[q * nb + b]) : 0.0;
    }
   }
  });
  return cs;
}

struct WalkStats {
  int64_t visited = 0;   // nodes given the opening test
  int64_t cut = 0;       // absorbing cells: accepted cells and opened leaves
  int64_t segments = 0;  // (beam, cut cell) pairs with a chord of positive length
  int64_t sources = 0;   // point sources added
};


template <class T>
struct Problem {
  const Tree* t;
  const Aggregates<T>* ag;
  const std::vector<T>* tab;  // [n][P][nb]
  const std::vector<T>* kappa;
  const std::vector<T>* lum;
  int nside;
  double theta;
  uint32_t flags;
  double h_default;
  std::vector<double> dirs;   // [npix][3]
  std::vector<int64_t> pair;  // [npix]
  std::vector<int64_t> leaf_of;  // [N] original index -> its leaf (FLAG_BUCKET)
  bool directed = false;         // R12: aim one beam at `target`
  double target[3] = {0, 0, 0};
  double tau_refine = std::numeric_limits<double>::infinity();  // R13
  const std::vector<double>* dtau = nullptr;                     // [nodes]
  const CsmTables* csm = nullptr;                                // R14
  std::vector<double> pp_r;                  // [nodes] r_pp of each leaf (FLAG_PP)
  std::vector<std::vector<int64_t>> pp_list; // [nodes] its p-p particles (original)
};

// R11: the p-p radius and particles of the bucket centred on xo whose box
// reaches r0 from its centre, by scanning every element.
inline double element_h(const Tree& t, int64_t j, double h_default) {
  return t.h.empty() ? h_default : t.h[j];
}

void pp_sphere(const Tree& t, const double xo[3], double r0, double beam, double h_default,
               double& rpp, std::vector<int64_t>& list) {
  auto dist = [&](int64_t j) {
    double s = 0.0;
    for (int a = 0; a < 3; ++a) {
      const double d = t.pos[3 * j + a] - xo[a];
      s += d * d;
    }
    return std::sqrt(s);
  };
  rpp = r0;
  for (int it = 0; it < 64; ++it) {
    double H = 0.0;
    for (int64_t j = 0; j < t.N; ++j)
      if (t.mass[j] > 0.0 && dist(j) < rpp) H = std::max(H, element_h(t, j, h_default));
    const double grown = std::max(rpp, H / beam);
    if (grown == rpp) break;
    rpp = grown;
  }
  list.clear();
  for (int64_t j = 0; j < t.N; ++j)
    if (t.mass[j] > 0.0 && dist(j) < rpp) list.push_back(j);
}

// J of one receiver, every band (Sec. 2.5).
template <class T>
void walk_receiver(const Problem<T>& pr, int64_t i_orig, T* Jout, WalkStats* st) {
  const Tree& t = *pr.t;
  const Aggregates<T>& ag = *pr.ag;
  const int nb = t.nb;
  const int64_t npix = 12 * static_cast<int64_t>(pr.nside) * pr.nside;
  const int64_t P = npix / 2;
  const double* xi = &t.pos[3 * i_orig];
  // R10: with per-bucket beams the walk's origin is the centre of the
  // receiver's leaf box, otherwise the receiver itself.
  double xo[3] = {xi[0], xi[1], xi[2]};
  if (pr.flags & FLAG_BUCKET) {
    double blo[3], bhi[3];
    node_box(t.nodes[pr.leaf_of[i_orig]], t.lo, t.size, blo, bhi);
    for (int a = 0; a < 3; ++a) xo[a] = 0.5 * (blo[a] + bhi[a]);
  }
  // R11: the bucket's p-p radius and particles
  const bool pp = (pr.flags & FLAG_PP) != 0;
  const double rpp = pp ? pr.pp_r[pr.leaf_of[i_orig]] : 0.0;
  const std::vector<int64_t>* pplist = pp ? &pr.pp_list[pr.leaf_of[i_orig]] : nullptr;
  // R12: the beam holding the target's direction points at the target
  std::vector<double> dirs_directed;
  const double* dirs = pr.dirs.data();
  if (pr.directed) {
    double vt[3], nt = 0.0;
    for (int a = 0; a < 3; ++a) {
      vt[a] = pr.target[a] - xo[a];
      nt += vt[a] * vt[a];
    }
    nt = std::sqrt(nt);
    if (nt > 0.0) {
      const int64_t kt = vec2pix_ring(pr.nside, vt);
      dirs_directed = pr.dirs;
      for (int a = 0; a < 3; ++a) dirs_directed[3 * kt + a] = vt[a] / nt;
      dirs = dirs_directed.data();
    }
  }
  struct CutCell {
    int64_t node;
    double lo[3], hi[3];
  };
  struct Src {
    T p[3];
    const T* L;         // nb luminosities
    int64_t elem = -1;  // the element, for a single-element source
    int64_t node = -1;  // the cell, for an accepted cell's source
  };
  std::vector<CutCell> cut;
  std::vector<Src> srcs;
  WalkStats ws;

  // Sec. 2.5.2: open iff d == 0 or B > theta d (d: distance to the closest
  // point of the cell; B: largest distance from the centre of luminosity to
  // the cell edge).  An accepted cell is one absorber and, if luminous, one
  // source at its centre of luminosity; an opened leaf is one absorber and
  // contributes its luminous elements one by one; an opened internal node
  // hands the test to its two halves.
  std::vector<int64_t> stack(1, 0);
  while (!stack.empty()) {
    int64_t q = stack.back();
    stack.pop_back();
    const Node& nd = t.nodes[q];
    CutCell cc;
    cc.node = q;
    node_box(nd, t.lo, t.size, cc.lo, cc.hi);
    ++ws.visited;
    bool open = cell_opens(xo, cc.lo, cc.hi, ag.B[q], pr.theta) ||
                (pp && box_distance(xo, cc.lo, cc.hi) < rpp) ||
                (pr.dtau && (*pr.dtau)[q] > pr.tau_refine);
    if (!open) {
      cut.push_back(cc);
      if (val(ag.Ltot[q]) > 0.0) {
        Src s;
        for (int a = 0; a < 3; ++a) s.p[a] = ag.c[3 * q + a];
        s.L = &ag.L[q * nb];
        s.node = q;
        srcs.push_back(s);
      }
    } else if (nd.child < 0) {
      cut.push_back(cc);
      for (int64_t e = nd.first; e < nd.first + nd.count; ++e) {
        int64_t j = t.perm[e];
        if (j == i_orig) continue;  // no self-illumination (Sec. 2.1)
        double lt = 0.0;
        for (int b = 0; b < nb; ++b) lt += val((*pr.lum)[j * nb + b]);
        if (!(lt > 0.0)) continue;
        Src s;
        for (int a = 0; a < 3; ++a) s.p[a] = T(t.pos[3 * j + a]);
        s.L = &(*pr.lum)[j * nb];
        s.elem = j;
        srcs.push_back(s);
      }
    } else {
      stack.push_back(nd.child + 1);
      stack.push_back(nd.child);
    }
  }
  ws.cut = static_cast<int64_t>(cut.size());

  // Chords of every beam with every absorbing cell of the cut (R5).
  struct Seg {
    double t0, t1;
    const T* alpha;  // nb values for this beam's direction pair
  };
  std::vector<std::vector<Seg>> segs(npix);
  for (int64_t k = 0; k < npix; ++k) {
    const double* nk = &dirs[3 * k];
    for (const CutCell& cc : cut) {
      double t0, t1;
      if (!ray_chord(xo, nk, cc.lo, cc.hi, t0, t1)) continue;
      if (pp) {  // R11: cells absorb only beyond r_pp
        t0 = std::max(t0, rpp);
        if (!(t1 > t0)) continue;
      }
      segs[k].push_back({t0, t1, &(*pr.tab)[(cc.node * P + pr.pair[k]) * nb]});
      ++ws.segments;
    }
  }

  // Sec. 2.5.1: a source joins the one beam holding its direction (from the
  // walk's origin); the optical depth along that beam up to the projected
  // distance s is scaled by r/s, r the receiver's distance to the source; the
  // source adds L e^{-tau} g(r) (R6, Eq. intint with SOFT).
  const double hi_ = t.h.empty() ? pr.h_default : t.h[i_orig];
  for (int b = 0; b < nb; ++b) Jout[b] = T(0.0);
  for (const Src& s : srcs) {
    T vo[3] = {s.p[0] - xo[0], s.p[1] - xo[1], s.p[2] - xo[2]};
    if (val(vo[0]) == 0.0 && val(vo[1]) == 0.0 && val(vo[2]) == 0.0) continue;
    double vv[3] = {val(vo[0]), val(vo[1]), val(vo[2])};
    int64_t k = vec2pix_ring(pr.nside, vv);
    const double* nk = &dirs[3 * k];
    T sp = vo[0] * nk[0] + vo[1] * nk[1] + vo[2] * nk[2];
    if (!(val(sp) > 0.0)) continue;  // cannot happen: beam radius < 90 degrees
    T v[3] = {s.p[0] - xi[0], s.p[1] - xi[1], s.p[2] - xi[2]};
    T r = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    if (val(r) == 0.0) continue;
    ++ws.sources;
    T g = (pr.flags & FLAG_SOFT) ? soft_kernel(r, hi_) : T(1.0) / (4.0 * kPi * r * r);
    // R11: the p-p particles in front of the receiver that cross the segment
    std::vector<T> taupp(nb, T(0.0));
    if (pp) {
      for (int64_t j : *pplist) {
        if (j == i_orig || j == s.elem) continue;
        const double* xj = &t.pos[3 * j];
        T dj[3] = {xj[0] - s.p[0], xj[1] - s.p[1], xj[2] - s.p[2]};
        T djs = sqrt(dj[0] * dj[0] + dj[1] * dj[1] + dj[2] * dj[2]);
        if (!(val(djs) < val(r))) continue;  // not closer to the source
        // distance from x_j to the segment x_i -> source
        T w[3] = {xj[0] - xi[0], xj[1] - xi[1], xj[2] - xi[2]};
        T tt = (w[0] * v[0] + w[1] * v[1] + w[2] * v[2]) / (r * r);
        if (val(tt) < 0.0) tt = T(0.0);
        if (val(tt) > 1.0) tt = T(1.0);
        T e[3] = {w[0] - tt * v[0], w[1] - tt * v[1], w[2] - tt * v[2]};
        T bj = sqrt(e[0] * e[0] + e[1] * e[1] + e[2] * e[2]);
        const double hj = element_h(t, j, pr.h_default);
        if (!(val(bj) < hj)) continue;
        T sigma = (3.0 * t.mass[j] / (kPi * hj * hj)) * (T(1.0) - bj / hj);
        for (int b = 0; b < nb; ++b) taupp[b] += (*pr.kappa)[j * nb + b] * sigma;
      }
    }
    // R14: a cell source's own ray replaces the beam beyond its projected edge
    T s_abs = sp;
    const double* tcsm = nullptr;
    if (pr.csm && s.node >= 0) {
      const int64_t ka = pr.csm->anti[k];
      const int64_t npx = static_cast<int64_t>(pr.dirs.size() / 3);
      s_abs = sp - pr.csm->d[s.node * npx + ka];
      if (val(s_abs) < 0.0) s_abs = T(0.0);
      tcsm = &pr.csm->tau[(s.node * npx + ka) * nb];
    }
    for (int b = 0; b < nb; ++b) {
      T tau = 0.0;
      for (const Seg& sg : segs[k]) {
        if (val(s_abs) <= sg.t0) continue;
        T len = (val(s_abs) < sg.t1) ? (s_abs - sg.t0) : T(sg.t1 - sg.t0);
        tau += sg.alpha[b] * len;
      }
      if (tcsm) tau += tcsm[b];
      tau = tau * (r / sp) + taupp[b];
      Jout[b] += s.L[b] * exp(-tau) * g;
    }
  }
  if (pr.flags & FLAG_THICK) {
    // Eq. taucorr with the element's own optical depth tau = alpha h,
    // alpha = kappa rho = kappa m / h^3.
    for (int b = 0; b < nb; ++b) {
      T taui = (*pr.kappa)[i_orig * nb + b] * t.mass[i_orig] / (hi_ * hi_);
      Jout[b] = Jout[b] * thick_factor(taui);
    }
  }
  if (st) *st = ws;
}

template <class T>
Problem<T> make_problem(const Tree& t, const Aggregates<T>& ag, const std::vector<T>& tab,
                        const std::vector<T>& kappa, const std::vector<T>& lum, int nside,
                        double theta, uint32_t flags) {
  Problem<T> pr;
  pr.t = &t;
  pr.ag = &ag;
  pr.tab = &tab;
  pr.kappa = &kappa;
  pr.lum = &lum;
  pr.nside = nside;
  pr.theta = theta;
  pr.flags = flags;
  int64_t ng = 0;
  for (int64_t i = 0; i < t.N; ++i) ng += (t.mass[i] > 0.0);
  pr.h_default = std::cbrt(t.size * t.size * t.size / static_cast<double>(std::max<int64_t>(ng, 1)));
  const int64_t npix = 12 * static_cast<int64_t>(nside) * nside;
  pr.dirs.resize(npix * 3);
  pr.pair.resize(npix);
  for (int64_t k = 0; k < npix; ++k) {
    pix2vec_ring(nside, k, &pr.dirs[3 * k]);
    pr.pair[k] = pair_of_pixel(nside, k);
  }
  if (flags & (FLAG_BUCKET | FLAG_PP)) {
    pr.leaf_of.assign(t.N, -1);
    for (size_t q = 0; q < t.nodes.size(); ++q) {
      const Node& nd = t.nodes[q];
      if (nd.child >= 0) continue;
      for (int64_t e = nd.first; e < nd.first + nd.count; ++e)
        pr.leaf_of[t.perm[e]] = static_cast<int64_t>(q);
    }
  }
  return pr;
}


// R11: r_pp and the p-p particles of every bucket that holds a receiver.
template <class T>
void prepare_pp(Problem<T>& pr, const int64_t* active, int64_t A, int nthreads) {
  if (!(pr.flags & FLAG_PP)) return;
  const Tree& t = *pr.t;
  pr.pp_r.assign(t.nodes.size(), 0.0);
  pr.pp_list.assign(t.nodes.size(), {});
  std::vector<char> seen(t.nodes.size(), 0);
  std::vector<int64_t> leaves;
  for (int64_t a = 0; a < A; ++a) {
    const int64_t q = pr.leaf_of[active[a]];
    if (!seen[q]) {
      seen[q] = 1;
      leaves.push_back(q);
    }
  }
  const int64_t npix = 12 * static_cast<int64_t>(pr.nside) * pr.nside;
  const double beam = std::sqrt(4.0 * kPi / static_cast<double>(npix));
  parallel_for(static_cast<int64_t>(leaves.size()), nthreads, [&](int64_t l) {
    const int64_t q = leaves[l];
    double blo[3], bhi[3], xo[3], r0 = 0.0;
    node_box(t.nodes[q], t.lo, t.size, blo, bhi);
    for (int a = 0; a < 3; ++a) {
      xo[a] = 0.5 * (blo[a] + bhi[a]);
      r0 += 0.25 * (bhi[a] - blo[a]) * (bhi[a] - blo[a]);
    }
    pp_sphere(t, xo, std::sqrt(r0), beam, pr.h_default, pr.pp_r[q], pr.pp_list[q]);
  });
}

struct OracleTree {
  Tree t;
  Aggregates<double> ag;
  std::vector<double> tab;
  int tab_nside = -1;
  bool tab_linear = false;
  double tau_refine = std::numeric_limits<double>::infinity();  // R13
  std::vector<double> dtau;                                      // [nodes]
  CsmTables csm;                                                 // R14
  int csm_nside = -1;
  bool csm_linear = false;
};

// R14: the complex source model for this nside and averaging, on first use.
void ensure_csm(OracleTree& ot, int nside, bool linear);

// R13: the optical-depth variation inside every cell, from the leaves up
// (children come after their parent in breadth-first order).
std::vector<double> tau_variation(const Tree& t, const Aggregates<double>& ag) {
  const int64_t n = static_cast<int64_t>(t.nodes.size());
  const int nb = t.nb;
  std::vector<double> amin(n * nb), amax(n * nb), out(n, 0.0);
  for (int64_t q = n - 1; q >= 0; --q) {
    const Node& nd = t.nodes[q];
    for (int b = 0; b < nb; ++b) {
      if (nd.child < 0) {
        amin[q * nb + b] = amax[q * nb + b] = ag.alpha[q * nb + b];
      } else {
        const int64_t c = nd.child;
        amin[q * nb + b] = std::min(amin[c * nb + b], amin[(c + 1) * nb + b]);
        amax[q * nb + b] = std::max(amax[c * nb + b], amax[(c + 1) * nb + b]);
      }
    }
    double lo[3], hi[3], side = 0.0, var = 0.0;
    node_box(nd, t.lo, t.size, lo, hi);
    for (int a = 0; a < 3; ++a) side = std::max(side, hi[a] - lo[a]);
    for (int b = 0; b < nb; ++b) var = std::max(var, amax[q * nb + b] - amin[q * nb + b]);
    out[q] = var * side;
  }
  return out;
}

// Problems built from an oracle tree see its refinement setting.
template <class T>
void apply_refine(const OracleTree& ot, Problem<T>& pr) {
  if (std::isfinite(ot.tau_refine)) {
    pr.tau_refine = ot.tau_refine;
    pr.dtau = &ot.dtau;
  }
}

void ensure_table(OracleTree& ot, int nside, bool linear = false) {
  if (ot.tab_nside == nside && ot.tab_linear == linear) return;
  ot.tab = alpha_tables(ot.t, ot.ag, nside, linear);
  ot.tab_nside = nside;
  ot.tab_linear = linear;
}

void ensure_csm(OracleTree& ot, int nside, bool linear) {
  ensure_table(ot, nside, linear);
  if (ot.csm_nside == nside && ot.csm_linear == linear) return;
  ot.csm = csm_tables(ot.t, ot.ag, ot.tab, nside);
  ot.csm_nside = nside;
  ot.csm_linear = linear;
}


bool valid_nside(int nside) { return nside >= 1 && nside <= 64 && (nside & (nside - 1)) == 0; }

}  // namespace

// ---------------------------------------------------------------------------
// C interface for the Python tests (ctypes).  All arrays are host arrays.
extern "C" {

int oracle_version(void) { return 1; }

void oracle_morton_keys(const double* pos, int64_t N, const double* lo, double size, uint64_t* out) {
  for (int64_t i = 0; i < N; ++i) out[i] = morton_key(&pos[3 * i], lo, size);
}

// Builds the tree.  box_lo == NULL or box_size <= 0 selects the automatic
// cube: lo = per-axis minimum, size = the largest extent (1 if all points
// coincide).  Returns NULL on invalid input.
void* oracle_tree_build(const double* pos, const double* mass, const double* kappa,
                        const double* lum, const double* h, int64_t N, int nb,
                        const double* box_lo, double box_size, int bucket) {
  if (N < 0 || nb < 1 || bucket < 1) return nullptr;
  auto* ot = new OracleTree();
  Tree& t = ot->t;
  t.N = N;
  t.nb = nb;
  t.bucket = bucket;
  t.pos.assign(pos, pos + 3 * N);
  t.mass.assign(mass, mass + N);
  t.kappa.assign(kappa, kappa + N * nb);
  t.lum.assign(lum, lum + N * nb);
  if (h) t.h.assign(h, h + N);
  if (box_lo && box_size > 0.0) {
    for (int a = 0; a < 3; ++a) t.lo[a] = box_lo[a];
    t.size = box_size;
  } else {
    double mn[3], mx[3];
    for (int a = 0; a < 3; ++a) {
      mn[a] = N ? pos[a] : 0.0;
      mx[a] = mn[a];
    }
    for (int64_t i = 0; i < N; ++i)
      for (int a = 0; a < 3; ++a) {
        mn[a] = std::min(mn[a], pos[3 * i + a]);
        mx[a] = std::max(mx[a], pos[3 * i + a]);
      }
    double ext = 0.0;
    for (int a = 0; a < 3; ++a) ext = std::max(ext, mx[a] - mn[a]);
    for (int a = 0; a < 3; ++a) t.lo[a] = mn[a];
    t.size = ext > 0.0 ? ext : 1.0;
  }
  build_tree(t);
  ot->ag = compute_aggregates<double>(t, t.kappa, t.lum);
  return ot;
}

void oracle_tree_free(void* h) { delete static_cast<OracleTree*>(h); }

int64_t oracle_tree_num_nodes(void* h) { return static_cast<int64_t>(static_cast<OracleTree*>(h)->t.nodes.size()); }

int oracle_tree_max_depth(void* h) { return static_cast<OracleTree*>(h)->t.max_depth; }

void oracle_tree_box(void* h, double* lo, double* size) {
  const Tree& t = static_cast<OracleTree*>(h)->t;
  for (int a = 0; a < 3; ++a) lo[a] = t.lo[a];
  *size = t.size;
}

// Any output pointer may be NULL.
void oracle_tree_export(void* h, uint64_t* keys_orig, int64_t* perm, uint64_t* prefix,
                        int32_t* depth, int64_t* first, int64_t* count, int64_t* child,
                        int64_t* parent, double* box /*[n][6] lo,hi*/) {
  const Tree& t = static_cast<OracleTree*>(h)->t;
  for (int64_t i = 0; i < t.N; ++i) {
    if (keys_orig) keys_orig[i] = t.key[i];
    if (perm) perm[i] = t.perm[i];
  }
  for (size_t q = 0; q < t.nodes.size(); ++q) {
    const Node& nd = t.nodes[q];
    if (prefix) prefix[q] = nd.prefix;
    if (depth) depth[q] = nd.depth;
    if (first) first[q] = nd.first;
    if (count) count[q] = nd.count;
    if (child) child[q] = nd.child;
    if (parent) parent[q] = nd.parent;
    if (box) node_box(nd, t.lo, t.size, &box[6 * q], &box[6 * q + 3]);
  }
}

void oracle_tree_aggregates(void* h, double* L, double* Ltot, double* c, double* B,
                            double* alpha_leaf) {
  const OracleTree& ot = *static_cast<OracleTree*>(h);
  const int64_t n = static_cast<int64_t>(ot.t.nodes.size());
  const int nb = ot.t.nb;
  for (int64_t q = 0; q < n; ++q) {
    for (int b = 0; b < nb; ++b) {
      if (L) L[q * nb + b] = ot.ag.L[q * nb + b];
      if (alpha_leaf) alpha_leaf[q * nb + b] = ot.ag.alpha[q * nb + b];
    }
    if (Ltot) Ltot[q] = ot.ag.Ltot[q];
    for (int a = 0; a < 3; ++a)
      if (c) c[3 * q + a] = ot.ag.c[3 * q + a];
    if (B) B[q] = ot.ag.B[q];
  }
}

// out: [n_nodes][6 nside^2][nb]
int oracle_alpha_table(void* h, int nside, int linear, double* out) {
  if (!valid_nside(nside)) return -1;
  OracleTree& ot = *static_cast<OracleTree*>(h);
  ensure_table(ot, nside, linear != 0);
  std::memcpy(out, ot.tab.data(), ot.tab.size() * sizeof(double));
  return 0;
}

void oracle_pix2vec(int nside, double* out) {
  const int64_t npix = 12 * static_cast<int64_t>(nside) * nside;
  for (int64_t p = 0; p < npix; ++p) pix2vec_ring(nside, p, &out[3 * p]);
}

void oracle_vec2pix(int nside, const double* v, int64_t n, int64_t* out) {
  for (int64_t i = 0; i < n; ++i) out[i] = vec2pix_ring(nside, &v[3 * i]);
}

int64_t oracle_pair_of_pixel(int nside, int64_t k) { return pair_of_pixel(nside, k); }

// Weights and chord of Eq. transmissionavg; geo = {V1, V2, V12, V, d}.
double oracle_transmission_alpha(const double* E, int axis, const double* n, double a1,
                                 double a2, double* geo) {
  TransGeo g = transmission_geometry(E, axis, n);
  if (geo) {
    geo[0] = g.V1;
    geo[1] = g.V2;
    geo[2] = g.V12;
    geo[3] = g.V;
    geo[4] = g.d;
  }
  return transmission_alpha<double>(a1, a2, g);
}

double oracle_soft_kernel(double r, double h) { return soft_kernel<double>(r, h); }

double oracle_thick_factor(double tau) { return thick_factor<double>(tau); }

// J[A][nb] for the receivers `active` (original indices).  stats may be
// NULL, else [A][4] = visited, cut, segments, sources.  Returns 0 or -1.
int oracle_J(void* h, const int64_t* active, int64_t A, int nside, double theta, uint32_t flags,
             double* J, int nthreads, int64_t* stats) {
  if (!valid_nside(nside) || !(theta > 0.0)) return -1;
  if ((flags & (FLAG_PP | FLAG_CSM)) && !(flags & FLAG_BUCKET)) return -1;
  OracleTree& ot = *static_cast<OracleTree*>(h);
  for (int64_t a = 0; a < A; ++a)
    if (active[a] < 0 || active[a] >= ot.t.N) return -1;
  ensure_table(ot, nside, (flags & FLAG_LINEAR) != 0);
  if (flags & FLAG_CSM) ensure_csm(ot, nside, (flags & FLAG_LINEAR) != 0);
  Problem<double> pr = make_problem<double>(ot.t, ot.ag, ot.tab, ot.t.kappa, ot.t.lum, nside,
                                            theta, flags);
  apply_refine(ot, pr);
  if (flags & FLAG_CSM) pr.csm = &ot.csm;
  prepare_pp(pr, active, A, nthreads);
  const int nb = ot.t.nb;
  parallel_for(A, nthreads, [&](int64_t a) {
    WalkStats ws;
    walk_receiver<double>(pr, active[a], &J[a * nb], &ws);
    if (stats) {
      stats[4 * a + 0] = ws.visited;
      stats[4 * a + 1] = ws.cut;
      stats[4 * a + 2] = ws.segments;
      stats[4 * a + 3] = ws.sources;
    }
  });
  return 0;
}

// J with directed rays (R12): the per-bucket walk (flags must hold
// FLAG_BUCKET) with the beam holding target[3] aimed at it.  Returns 0 or -1.
int oracle_J_directed(void* h, const int64_t* active, int64_t A, int nside, double theta,
                      uint32_t flags, const double* target, double* J, int nthreads) {
  if (!valid_nside(nside) || !(theta > 0.0) || !(flags & FLAG_BUCKET)) return -1;
  OracleTree& ot = *static_cast<OracleTree*>(h);
  for (int64_t a = 0; a < A; ++a)
    if (active[a] < 0 || active[a] >= ot.t.N) return -1;
  ensure_table(ot, nside, (flags & FLAG_LINEAR) != 0);
  if (flags & FLAG_CSM) ensure_csm(ot, nside, (flags & FLAG_LINEAR) != 0);
  Problem<double> pr = make_problem<double>(ot.t, ot.ag, ot.tab, ot.t.kappa, ot.t.lum, nside,
                                            theta, flags);
  apply_refine(ot, pr);
  if (flags & FLAG_CSM) pr.csm = &ot.csm;
  pr.directed = true;
  for (int a = 0; a < 3; ++a) pr.target[a] = target[a];
  prepare_pp(pr, active, A, nthreads);
  const int nb = ot.t.nb;
  parallel_for(A, nthreads, [&](int64_t a) {
    walk_receiver<double>(pr, active[a], &J[a * nb], nullptr);
  });
  return 0;
}

// Forward-mode derivative of J[A][nb] with respect to one input:
// which = 0: kappa[elem][band], which = 1: lum[elem][band].  The cut, the
// beams and the tree stay those of the primal inputs.
int oracle_J_deriv(void* h, const int64_t* active, int64_t A, int nside, double theta,
                   uint32_t flags, int which, int64_t elem, int band, double* dJ, int nthreads) {
  if (!valid_nside(nside) || !(theta > 0.0) || (flags & FLAG_CSM)) return -1;
  if ((flags & FLAG_PP) && !(flags & FLAG_BUCKET)) return -1;
  OracleTree& ot = *static_cast<OracleTree*>(h);
  const Tree& t = ot.t;
  const int nb = t.nb;
  if (elem < 0 || elem >= t.N || band < 0 || band >= nb || (which != 0 && which != 1)) return -1;
  std::vector<Dual> kappa(t.kappa.begin(), t.kappa.end());
  std::vector<Dual> lum(t.lum.begin(), t.lum.end());
  if (which == 0) kappa[elem * nb + band].d = 1.0;
  else lum[elem * nb + band].d = 1.0;
  Aggregates<Dual> ag = compute_aggregates<Dual>(t, kappa, lum);
  std::vector<Dual> tab = alpha_tables<Dual>(t, ag, nside, (flags & FLAG_LINEAR) != 0);
  Problem<Dual> pr = make_problem<Dual>(t, ag, tab, kappa, lum, nside, theta, flags);
  apply_refine(ot, pr);
  prepare_pp(pr, active, A, nthreads);
  parallel_for(A, nthreads, [&](int64_t a) {
    std::vector<Dual> Jd(nb);
    walk_receiver<Dual>(pr, active[a], Jd.data(), nullptr);
    for (int b = 0; b < nb; ++b) dJ[a * nb + b] = Jd[b].d;
  });
  return 0;
}

// R11: r_pp and the p-p particles (original indices, sorted) of the leaf
// holding element i for this nside; list may be NULL (count only).
// Returns the number of particles, or -1.
int64_t oracle_pp_sphere(void* h, int64_t i, int nside, double* rpp, int64_t* list) {
  OracleTree& ot = *static_cast<OracleTree*>(h);
  const Tree& t = ot.t;
  if (i < 0 || i >= t.N || !valid_nside(nside)) return -1;
  Problem<double> pr = make_problem<double>(t, ot.ag, ot.tab, t.kappa, t.lum, nside, 1.0,
                                            FLAG_BUCKET | FLAG_PP);
  prepare_pp(pr, &i, 1, 1);
  const int64_t q = pr.leaf_of[i];
  *rpp = pr.pp_r[q];
  std::vector<int64_t> l = pr.pp_list[q];
  std::sort(l.begin(), l.end());
  if (list) std::copy(l.begin(), l.end(), list);
  return static_cast<int64_t>(l.size());
}

// R14: the complex source model's d [n][npix] and tau [n][npix][nb] for
// this nside and averaging (linear != 0).  Returns 0 or -1.
int oracle_csm_tables(void* h, int nside, int linear, double* d, double* tau) {
  OracleTree& ot = *static_cast<OracleTree*>(h);
  if (!valid_nside(nside)) return -1;
  ensure_csm(ot, nside, linear != 0);
  std::copy(ot.csm.d.begin(), ot.csm.d.end(), d);
  std::copy(ot.csm.tau.begin(), ot.csm.tau.end(), tau);
  return 0;
}

// R13: refinement for every later call; tau_refine <= 0 or NaN is
// rejected (-1), +infinity turns it off.  dtau_out (may be NULL) receives
// the per-node variation [nodes].
int oracle_set_tau_refine(void* h, double tau_refine, double* dtau_out) {
  OracleTree& ot = *static_cast<OracleTree*>(h);
  if (!(tau_refine > 0.0)) return -1;
  if (ot.dtau.empty()) ot.dtau = tau_variation(ot.t, ot.ag);
  ot.tau_refine = tau_refine;
  if (dtau_out) std::copy(ot.dtau.begin(), ot.dtau.end(), dtau_out);
  return 0;
}

// Opening decision for one cell with the given centre of luminosity.
int oracle_cell_opens(const double* blo, const double* bhi, const double* c, const double* x,
                      double theta, double* B_out) {
  double B = max_corner_distance(c, blo, bhi);
  if (B_out) *B_out = B;
  return cell_opens(x, blo, bhi, B, theta) ? 1 : 0;
}

// Optical depth along beam k of receiver i from 0 to s, band b, as the walk
// computes it (sum over the cut of alpha times the clipped chord), without
// the r/s correction.
double oracle_beam_tau(void* h, int64_t i_orig, int nside, double theta, int64_t k, double s,
                       int band) {
  OracleTree& ot = *static_cast<OracleTree*>(h);
  const Tree& t = ot.t;
  ensure_table(ot, nside);
  const int nb = t.nb;
  const int64_t P = 6 * static_cast<int64_t>(nside) * nside;
  const double* xi = &t.pos[3 * i_orig];
  double nk[3];
  pix2vec_ring(nside, k, nk);
  int64_t pk = pair_of_pixel(nside, k);
  double tau = 0.0;
  std::vector<int64_t> stack(1, 0);
  while (!stack.empty()) {
    int64_t q = stack.back();
    stack.pop_back();
    const Node& nd = t.nodes[q];
    double lo[3], hi[3];
    node_box(nd, t.lo, t.size, lo, hi);
    bool open = cell_opens(xi, lo, hi, ot.ag.B[q], theta) ||
                (std::isfinite(ot.tau_refine) && ot.dtau[q] > ot.tau_refine);
    if (open && nd.child >= 0) {
      stack.push_back(nd.child + 1);
      stack.push_back(nd.child);
      continue;
    }
    double t0, t1;
    if (!ray_chord(xi, nk, lo, hi, t0, t1)) continue;
    double len = std::max(0.0, std::min(t1, s) - t0);
    tau += ot.tab[(q * P + pk) * nb + band] * len;
  }
  return tau;
}

}  // extern "C"
