// Internal declarations of the GB300 TREVR2 library (not part of the ABI).
//
// Coordinates: everything on the device lives in the normalised root cube
// [0,1)^3 (u = (x - lo)/size, computed in FP64).  Cell boxes are then exact
// dyadic numbers in FP32; absorption is stored per normalised length
// (alpha * size) and J is rescaled by 1/size^2 at the end.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "trevr2.h"

namespace trevr2 {

constexpr int kMaxDepth = 63;
constexpr int kKeyBits = 21;

// ---------------------------------------------------------------------------
// Node record read by the walk: 32 bytes = two 16-byte loads.
struct __align__(16) NodeW {
  float lo[3];    // normalised lower corner (exact)
  float B;        // largest distance from the centre of luminosity to a corner
  int child;      // lower child, upper = child + 1; -1 for a leaf
  int aux;        // internal: row of the alpha table; leaf: first element (sorted)
  int count;      // elements under the node
  uint32_t meta;  // depth | flags
};
constexpr uint32_t kMetaDepthMask = 63u;
constexpr uint32_t kMetaLeaf = 1u << 8;
constexpr uint32_t kMetaHasL = 1u << 9;      // some luminosity below
constexpr uint32_t kMetaHasAlpha = 1u << 10; // some absorption below
constexpr int kMetaAxisShift = 12;            // split axis (depth mod 3) in bits 12-13
constexpr uint32_t kMetaChild0Alpha = 1u << 14;  // lower half has some absorption
constexpr uint32_t kMetaChild1Alpha = 1u << 15;  // upper half has some absorption

// Source found by the cut, binned to its beam: projected distance s along
// the beam, r/s, the geometric kernel g(r), and where its luminosity lives.
struct __align__(16) SrcEntry {
  float s;
  float rs;
  float w;
  int ref;  // node index, or sorted element index | kRefElement
};
constexpr int kRefElement = int(0x80000000u);

// Device status bits (OR-ed into the tree's status word).
constexpr uint32_t kStatusBadActive = 1u << 0;
constexpr uint32_t kStatusStackOverflow = 1u << 1;
constexpr uint32_t kStatusBadInput = 1u << 2;
constexpr uint32_t kStatusOutsideBox = 1u << 3;
constexpr uint32_t kStatusPPOverflow = 1u << 5;  // a p-p sphere held too many particles

// Geometry of the transmission average for one cell shape and one beam pair:
// weights V1/V (= V2/V), V12/V and the chord through the centre of a cell of
// unit scale (d scales with the cell, the weights do not).
struct __align__(16) TransGeo {
  float w1;
  float w12;
  float d_unit;
  float pad;
};

struct Table {
  int nside = 0;
  bool linear = false;         // linear absorption average instead of Eq. transmissionavg
  float* alpha = nullptr;      // [n_internal][P][nbp] normalised absorption
  float4* dirs = nullptr;      // [npix] beam directions (xyz), w = pair index (int bits)
  double* dirs64 = nullptr;    // [npix][3]
  TransGeo* geo = nullptr;     // [3][P]
  // complex source model (Sec. 2.7), built on first use with TREVR2_CSM
  float* csm_tau = nullptr;    // [n][npix][nbp] optical depth of each luminous cell's ray
  float* csm_d = nullptr;      // [n][npix] its length (normalised)
  int* csm_anti = nullptr;     // [npix] pixel of -n_k
};

// ---------------------------------------------------------------------------
struct Tree {
  int64_t N = 0;
  int nb = 0;
  int nbp = 0;     // bands padded to 1, 2 or 4
  int bucket = 12;
  double lo[3] = {0, 0, 0};
  double size = 1.0;
  int64_t n_nodes = 0;
  int64_t n_internal = 0;
  int max_depth = 0;
  bool has_h = false;
  cudaStream_t last_stream = nullptr;

  // elements, sorted by key
  uint64_t* keys = nullptr;   // [N]
  int* perm = nullptr;        // [N] sorted -> caller index
  int* inv = nullptr;         // [N] caller index -> sorted
  double* pos64 = nullptr;    // [N][3] normalised
  float4* pos32 = nullptr;    // [N] normalised xyz, w = total luminosity
  float* Lelem = nullptr;     // [N][nbp]
  float* km = nullptr;        // [N][nbp] kappa * m (caller units)
  float* hn = nullptr;        // [N] element size / size
  float* mass = nullptr;      // [N] element mass (caller units)

  // nodes (breadth first)
  uint64_t* prefix = nullptr; // [n]
  int* depth = nullptr;       // [n]
  int* first = nullptr;       // [n]
  int* count = nullptr;       // [n]
  int* child = nullptr;       // [n]
  int* parent = nullptr;      // [n]
  int* int_index = nullptr;   // [n] row in the alpha table, -1 for leaves
  NodeW* nodes = nullptr;     // [n]
  float* Lnode = nullptr;     // [n][nbp]
  float4* csrc = nullptr;     // [n] centre of luminosity (normalised) xyz, w = total L
  double* c64 = nullptr;      // [n][3] normalised centre of luminosity
  double* B64 = nullptr;      // [n] normalised B
  float* alpha_leaf = nullptr;// [n][nbp] normalised bucket absorption (0 internal)
  // refinement tau_refine (Sec. 2.5.2): node records with B raised where the
  // optical depth varies by more than tau_refine inside the cell
  float* dtau = nullptr;          // [n] optical-depth variation of each cell
  NodeW* nodes_refined = nullptr; // [n], kept until the tree is freed
  bool refine_on = false;
  double tau_refine = 0.0;
  std::vector<int64_t> level_begin;  // host: first node of each depth, plus end

  std::vector<Table> tables;  // cached per nside

  // walk buffers (grown on demand)
  void* scratch = nullptr;
  size_t scratch_bytes = 0;
  void* order_buf = nullptr;   // receivers in key order: keys + slots
  size_t order_bytes = 0;
  uint32_t* status = nullptr;             // device status word
  unsigned long long* counter = nullptr;  // device work counter
};

// ---------------------------------------------------------------------------
// Host helpers (errors, allocation).
void set_error(const char* fmt, ...);
void clear_error();

int cuda_fail(cudaError_t e, const char* what);

// Counts kernels launched by this library (host side; see trevr2_kernel_launches).
void note_launch();
#define T2_CUDA(call)                                            \
  do {                                                           \
    cudaError_t e_ = (call);                                     \
    if (e_ != cudaSuccess) return ::trevr2::cuda_fail(e_, #call);\
  } while (0)
#define T2_CHECK(rc_expr)        \
  do {                           \
    int rc_ = (rc_expr);         \
    if (rc_ != TREVR2_OK) return rc_; \
  } while (0)

// Every device allocation of the library (stream ordered, freed with
// dfree / cudaFreeAsync).  `what` names it in the error message.  A failure
// requested with trevr2_debug_set(TREVR2_DEBUG_FAIL_ALLOC, n) happens here.
int device_alloc(void** p, size_t bytes, cudaStream_t st, const char* what);

template <class T>
int dalloc(T** p, size_t count, cudaStream_t st) {
  if (count == 0) count = 1;
  return device_alloc(reinterpret_cast<void**>(p), count * sizeof(T), st, "device allocation");
}

template <class T>
void dfree(T*& p, cudaStream_t st) {
  if (p) cudaFreeAsync(p, st);
  p = nullptr;
}

// A temporary device buffer freed (stream ordered) when it goes out of
// scope, so that every early error return releases it.
template <class T>
struct DeviceTemp {
  T* p = nullptr;
  cudaStream_t st;
  explicit DeviceTemp(cudaStream_t s) : st(s) {}
  ~DeviceTemp() { dfree(p, st); }
  DeviceTemp(const DeviceTemp&) = delete;
  DeviceTemp& operator=(const DeviceTemp&) = delete;
};

// Capacity of the source cut's traversal stack set by
// trevr2_debug_set(TREVR2_DEBUG_SOURCE_STACK, c); 0 when not set.
int debug_source_stack_cap();

// Exclusive scan of n int32 values in place; *d_total (device) gets the sum.
// ws (device, scan_ws_ints(n) ints) or NULL to allocate one stream ordered.
size_t scan_ws_ints(int64_t n);
int scan_exclusive_i32(int* d, int64_t n, int* d_total, cudaStream_t st, int* ws = nullptr);

// Stable LSD radix sort of keys below 2^key_bits with int32 payload (in place).
// ws (device, radix_ws_bytes(n) bytes) or NULL to allocate one stream ordered.
size_t radix_ws_bytes(int64_t n);
int radix_sort_u64_i32(uint64_t* keys, int* vals, int64_t n, cudaStream_t st, int key_bits = 64,
                       void* ws = nullptr);

// Alpha tables and beam directions for one nside and averaging (built and
// cached): Eq. transmissionavg, or with `linear` the volume-weighted linear
// average of the halves (Sec. 2.6's comparison scheme).
int ensure_table(Tree* t, int nside, cudaStream_t st, Table** out, bool linear = false);

inline int nbp_of(int nb) { return nb <= 1 ? 1 : (nb == 2 ? 2 : 4); }

// Extent of a cell at `depth` along axis a: 2^-(number of splits on a).
__host__ __device__ inline int splits_on_axis(int depth, int a) { return (depth + 2 - a) / 3; }

}  // namespace trevr2
