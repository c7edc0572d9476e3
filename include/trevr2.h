/*
 * trevr2.h — C ABI of the GB300 TREVR2 reverse-ray-trace library.
 *
 * The method is TREVR2 (Wadsley, Baumschlager & Shen, arXiv:2310.15235):
 * for every active receiving element, rays leave along the HEALPix beam
 * directions (Sec. 1.3, Sec. 2.5) through a binary radiation tree (Sec. 2.3),
 * accumulating optical depth from cells whose absorption is the
 * transmission average of their halves (Sec. 2.6, Eq. transmissionavg),
 * and adding every source cell accepted by the opening criterion B/d > theta
 * (Sec. 2.5.2), attenuated by e^{-tau} with tau taken along its beam to the
 * projected distance and scaled by r/s (Sec. 2.5.1).  The result is the
 * integrated intensity J = integral of I over solid angle, per receiver and
 * band, whose far-field kernel is L/(4 pi r^2) (Eq. intint).
 *
 * Conventions for every entry point:
 *  - Array arguments are DEVICE pointers unless marked "host", contiguous,
 *    row-major, in the units of the caller (positions in any length unit;
 *    J comes back in luminosity per length^2).
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream).  All work
 *    is stream ordered; inputs may be released once the stream has passed
 *    the call.
 *  - The return value is TREVR2_OK (0) or a negative TREVR2_E* code; the
 *    message of the last error on the calling thread is trevr2_last_error().
 *    No C++ exception crosses this boundary and no kernel traps: device-side
 *    problems are recorded in a status word and reported as error codes.
 *  - Calls that use one tree must not overlap on the GPU (one stream, or
 *    ordered by events): the tree owns one set of walk buffers.
 */
#ifndef TREVR2_H
#define TREVR2_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
#define TREVR2_OK 0
#define TREVR2_EINVAL (-1)      /* invalid argument or input value            */
#define TREVR2_ENOMEM (-2)      /* device or host allocation failed           */
#define TREVR2_ECUDA (-3)       /* a CUDA runtime call failed                 */
#define TREVR2_ETIMEOUT (-4)    /* reserved: no kernel of this library waits on
                                   the device, so no call returns it           */
#define TREVR2_EUNSUPPORTED (-5)/* outside the supported sizes (see below)    */
#define TREVR2_EINTERNAL (-6)   /* an internal capacity check failed          */

/* Flags of trevr2_J. */
#define TREVR2_SOFT 1u   /* finite-size element kernel, Eq. intint (Sec. 2.2)   */
#define TREVR2_THICK 2u  /* optically thick element factor, Eq. taucorr (Sec. 2.1) */
#define TREVR2_ASYNC 4u  /* do not synchronise; check later with trevr2_status */
#define TREVR2_LINEAR 8u /* internal cells take the volume-weighted linear average of
                            their halves' absorption, the scheme Sec. 2.6 compares
                            Eq. transmissionavg with (direction independent) */
#define TREVR2_BUCKET 16u /* per-bucket beams (Sec. 2, Sec. 2.5.1): one walk per
                             leaf holding receivers, from its box centre; each
                             receiver scales the beam optical depth by its own
                             distance over the projected one (trevr2_J only) */
#define TREVR2_PP 32u    /* with TREVR2_BUCKET: particle-particle absorption inside
                            the bucket's p-p radius (Sec. 2.4; trevr2_J only) */
#define TREVR2_CSM 64u   /* with TREVR2_BUCKET: the complex source model (Sec. 2.7,
                            Eq. srccomb; trevr2_J and trevr2_J_directed only) */

/* Supported sizes: 1 <= nb <= 4 bands; nside a power of two in [1, 16];
 * N < 2^31 elements; 1 <= bucket <= 4096. */
#define TREVR2_MAX_BANDS 4
#define TREVR2_MAX_NSIDE 16

typedef struct trevr2_tree trevr2_tree;

/*
 * trevr2_build — the radiation tree of Sec. 2.3 with the per-cell
 * quantities of Sec. 2.6 and Fig. sourcecombine (summed luminosity per band,
 * centre of luminosity, bucket absorption sum(kappa m)/V_box).
 *
 *  pos     [N][3] float64  element positions
 *  mass    [N]    float32  element masses (0 for pure point sources)
 *  kappa   [N][nb] float32 opacity per unit mass, per band
 *  lum     [N][nb] float32 luminosity per band
 *  h       [N]    float32  element size (m/rho)^(1/3), used by TREVR2_SOFT and
 *                          TREVR2_THICK; NULL = (V_root / N_gas)^(1/3)
 *  N, nb   element and band counts (1 <= nb <= TREVR2_MAX_BANDS)
 *  box_lo  host [3] lower corner of the root cube and box_size its edge;
 *          box_lo == NULL or box_size <= 0 picks the bounding cube of the
 *          positions (lo = per-axis minimum, edge = largest extent).  With an
 *          explicit cube every position must lie inside it.
 *  bucket  largest element count of a leaf (paper default 12)
 *  out     receives the new tree; the tree owns its device memory until
 *          trevr2_free.  The tree is geometric cyclic x,y,z bisection of
 *          63-bit Morton keys; nodes are numbered breadth first, by key prefix
 *          within a depth.
 * Errors: EINVAL for NULL pointers, N < 0, nb out of range, non-finite
 * positions, negative or non-finite mass/kappa/lum/h, positions outside an
 * explicit cube; ENOMEM; ECUDA.  This call synchronises `stream`.
 */
int trevr2_build(const double* pos, const float* mass, const float* kappa, const float* lum,
                 const float* h, int64_t N, int nb, const double* box_lo, double box_size,
                 int bucket, void* stream, trevr2_tree** out);

/*
 * trevr2_J — integrated intensity J per active receiver and band
 * (Sec. 2.5: cell opening B/d > theta, HEALPix beams with N_ray = 12 nside^2,
 * transmission-averaged optical depth to each source's projected distance
 * corrected by r/s, no self-illumination).
 *
 *  active  [A] int64  receiver indices in the caller's element order
 *  nside   HEALPix resolution (power of two, 1..TREVR2_MAX_NSIDE); the alpha
 *          tables for a new nside (and averaging) are built on first use
 *          and cached
 *  theta   opening parameter theta_rad > 0 (paper default 0.75)
 *  bands   host [nbsel] band indices to return, or NULL = all nb bands
 *  flags   TREVR2_SOFT | TREVR2_THICK | TREVR2_LINEAR | TREVR2_BUCKET |
 *          TREVR2_PP | TREVR2_CSM | TREVR2_ASYNC.  With TREVR2_BUCKET the cut, the beam of each source,
 *          its projected distance s and the optical depth to s are those of
 *          the centre of the leaf box holding the receiver, shared by every
 *          receiver of that leaf; each receiver adds L g(r) e^{-tau r/s} with
 *          r its own distance to the source (its own h and Eq. taucorr
 *          factor under TREVR2_SOFT / TREVR2_THICK).  A source exactly at a
 *          bucket centre has no beam and is skipped.  TREVR2_PP (needs
 *          TREVR2_BUCKET, else EINVAL) adds Sec. 2.4: the bucket's p-p radius
 *          r_pp starts at the sphere through its box corners and grows until
 *          no gas element (m > 0) inside is wider than the beam there
 *          (h <= r_pp sqrt(4 pi / N_ray)); cells within r_pp open, cell
 *          absorption counts beyond r_pp only, and every p-p particle k
 *          (not the receiver, not the source) closer to the source than the
 *          receiver and within h_k of the segment (distance b) adds
 *          kappa_k 3 m_k (1 - b / h_k) / (pi h_k^2).  A sphere holding more
 *          than 4096 particles gives EUNSUPPORTED.  TREVR2_CSM (needs
 *          TREVR2_BUCKET, else EINVAL) adds Sec. 2.7: every luminous cell
 *          keeps, per HEALPix direction, the ray from its centre of
 *          luminosity to its box edge (leaves: bucket alpha times length;
 *          parents: the children's rays clipped or extended, through the
 *          sibling, to the parent's end plane and combined by Eq. srccomb),
 *          built per nside and averaging on first use ([nodes][N_ray] per
 *          band and length); an accepted cell's source then takes the beam
 *          only up to its projected edge s - d and adds its own ray towards
 *          the bucket.  Batch plans take TREVR2_BUCKET with or without
 *          TREVR2_PP and TREVR2_CSM.  trevr2_J_backward returns EUNSUPPORTED
 *          for any of the three and trevr2_J_noalloc EINVAL (an unknown flag
 *          bit there).
 *  J       [A][nbsel] float32 output, overwritten
 * Active indices outside [0, N) give EINVAL (their rows are set to NaN).
 * Without TREVR2_ASYNC the call synchronises `stream` and returns any device
 * status; with it the call returns after enqueueing and trevr2_status
 * reports the device status later.
 */
int trevr2_J(trevr2_tree* tree, const int64_t* active, int64_t A, int nside, float theta,
             const int* bands, int nbsel, uint32_t flags, float* J, void* stream);

/*
 * trevr2_J_directed — trevr2_J with one beam aimed at a target (Sec. 3.4.1:
 * for a single-source test the beam is pointed at the source instead of along
 * the centre of its HEALPix pixel).  Per bucket, the beam whose pixel holds
 * the direction from the bucket centre to `target` takes that exact
 * direction; it keeps its pixel's direction pair for the cells' absorption,
 * and the sources binned into it take their projected distance along it.
 * A target at a bucket centre leaves that bucket's beams as they are.
 *
 *  target  host [3] float64 point in the caller's coordinates
 * The other arguments, the output and the errors are those of trevr2_J;
 * flags must include TREVR2_BUCKET (else EINVAL), as must a NULL or
 * non-finite target.
 */
int trevr2_J_directed(trevr2_tree* tree, const int64_t* active, int64_t A, int nside, float theta,
                      const int* bands, int nbsel, uint32_t flags, const double* target,
                      float* J, void* stream);

/*
 * trevr2_set_tau_refine — absorption refinement (Sec. 2.5.2, the TREVR
 * criterion the paper keeps as an option, off by default): every later walk
 * on this tree also opens a cell whose optical depth varies by more than
 * tau_refine inside it, the variation being (largest - smallest bucket alpha
 * among the leaves under the cell, per band) times the cell's longest side,
 * the largest over the bands.  Leaves do not open further.  Applies to
 * trevr2_J, trevr2_J_directed, trevr2_J_noalloc and trevr2_J_backward, and
 * to batch plans created while it is on (they read the tree's refined node
 * copy when they run; create plans after setting it).
 *
 *  tau_refine  > 0; +infinity turns refinement off (the default)
 * The first call allocates the per-cell variation and a copy of the node
 * records (freed by trevr2_free).  Stream ordered, does not synchronise.
 * Errors: EINVAL (NULL tree, tau_refine <= 0 or NaN), ENOMEM, ECUDA.
 */
int trevr2_set_tau_refine(trevr2_tree* tree, double tau_refine, void* stream);

/*
 * trevr2_prepare — builds and caches the per-direction absorption tables of
 * Eq. transmissionavg (Sec. 2.6; N_ray/2 values per cell and band) and the
 * HEALPix beam table for `nside`, without running a walk.  trevr2_J does the
 * same on first use of an nside; calling this first keeps that work out of
 * a later trevr2_J.  The linear-average tables (TREVR2_LINEAR) are built by
 * the first call that asks for them.  Stream ordered, does not synchronise.
 * Errors: EINVAL (NULL tree, bad nside), ENOMEM, ECUDA.
 */
int trevr2_prepare(trevr2_tree* tree, int nside, void* stream);

/*
 * trevr2_J_noalloc — trevr2_J without any device allocation.  The paper has
 * no counterpart: this entry point exists for callers that cannot let a
 * library allocate device memory (host codes that own all device memory
 * through their own arena or a fixed budget, or that call from a context
 * where an allocation could block or fail).
 *
 * Arguments, output and errors are those of trevr2_J, with two differences:
 *  - the tables for `nside` must already exist (trevr2_prepare, or an
 *    earlier trevr2_J with the same nside; with TREVR2_LINEAR an earlier
 *    trevr2_J with that flag); otherwise EINVAL;
 *  - the walk buffers live in one fixed 16 MiB device array inside the
 *    library (256 source records per warp and pass, which caps the grid at
 *    1,820 resident warps).  The walk loops over receivers and makes more
 *    passes when a receiver has more sources, so any A works; a launch that
 *    would need more than the array holds is rejected with EUNSUPPORTED.
 * Every process that loads the library holds that array on each GPU it uses
 * until it exits.  All calls share the array: calls whose work overlaps on
 * the GPU (on any tree, from any thread or stream) race and must be ordered
 * by the caller.  Every call looks up the array's device address
 * (cudaGetSymbolAddress) with the tree's device current, so the address
 * stays right if the device's context is reset; the first call on a device
 * also loads the library's module there, so make that first call before any
 * stream capture.
 */
int trevr2_J_noalloc(trevr2_tree* tree, const int64_t* active, int64_t A, int nside, float theta,
                     const int* bands, int nbsel, uint32_t flags, float* J, void* stream);

/*
 * trevr2_J_backward — adjoint of trevr2_J: for a loss whose gradient with
 * respect to J is gJ, returns dLoss/dkappa and dLoss/dlum of every element.
 * It differentiates the same map as trevr2_J with the discrete choices held
 * fixed (tree, cut of Sec. 2.5.2, beam of every source): through the
 * attenuation e^{-tau} of every source along its beam (Sec. 2.5.1), the
 * transmission average of the per-direction absorption (Sec. 2.6,
 * Eq. transmissionavg) down to the bucket absorption sum(kappa m)/V_box of
 * the leaves, the cell luminosities and their centres of luminosity, and,
 * with TREVR2_THICK, the receiver's own Eq. taucorr factor.  The traversals
 * are walked again; nothing from the forward call is kept.
 *
 *  active, A, nside, theta, bands, nbsel, flags   as for trevr2_J
 *  gJ       [A][nbsel] float32 dLoss/dJ (rows and columns as trevr2_J's J)
 *  g_kappa  [N][nb] float32 output dLoss/dkappa in the caller's element
 *           order (the units of J per unit kappa), overwritten
 *  g_lum    [N][nb] float32 output dLoss/dlum, overwritten
 * Positions, masses and sizes are not differentiated.  The call allocates
 * its gradient buffers (about the size of the alpha table for nside plus
 * 8 nb floats per element) stream ordered and frees them before returning.
 * Errors: as trevr2_J (EINVAL, EUNSUPPORTED, ENOMEM, ECUDA).  Without
 * TREVR2_ASYNC the call synchronises `stream` and returns the device status.
 */
int trevr2_J_backward(trevr2_tree* tree, const int64_t* active, int64_t A, int nside, float theta,
                      const int* bands, int nbsel, uint32_t flags, const float* gJ,
                      float* g_kappa, float* g_lum, void* stream);

/* ---- Batches: many receiver subsets over several trees -------------- */

/*
 * With individual timesteps (Sec. 1.2) only the elements on the current rung
 * need J, so one step asks for many small receiver subsets; Sec. 3.1 runs
 * several independent snapshots.  A batch walks all of them in one persistent
 * launch: subsets s = 0..nsub-1 are concatenated, subset s owning rows
 * offsets[s] <= r < offsets[s+1] of `active` and of J, and walked in tree
 * trees[tree_of[s]].  Each row equals what trevr2_J gives for the same tree,
 * receiver, nside, theta and flags (all nb bands, in band order), bit for
 * bit.  Rows asking for the same receiver of the same tree (in one subset or
 * in several) are walked once and copied: a run sorts the rows by (tree,
 * receiver position in the tree's Morton order), walks the distinct ones in
 * that order and scatters the results.  With TREVR2_BUCKET (the paper's own
 * per-bucket beams, Sec. 2.5.1; optionally with TREVR2_PP and TREVR2_CSM) a
 * run walks every distinct (tree, bucket) once, from the bucket centre, for
 * all the distinct receivers of that bucket that any subset asks for: each
 * row still equals trevr2_J's row for the same tree, receiver and flags.
 */
typedef struct trevr2_batch trevr2_batch;

/* Most trees in one batch. */
#define TREVR2_MAX_BATCH_TREES 32

/*
 * trevr2_batch_create — a reusable batch plan.
 *  trees    host [ntrees] trees with the same band count nb
 *           (1 <= ntrees <= TREVR2_MAX_BATCH_TREES); they must outlive the
 *           plan and must not be rebuilt while it exists
 *  offsets  host [nsub + 1] int64, offsets[0] = 0, non-decreasing
 *  tree_of  host [nsub] int, tree index of each subset
 *  nside, theta, flags   as for trevr2_J (TREVR2_ASYNC is ignored here);
 *           TREVR2_PP and TREVR2_CSM need TREVR2_BUCKET (else EINVAL).  A
 *           plan with TREVR2_PP holds the p-p particle arrays of every
 *           resident warp (about 208 KiB each); with TREVR2_CSM creation
 *           builds the trees' complex-source tables for `nside`
 *  out      receives the plan.  Creation builds any missing alpha tables of
 *           the trees for `nside`, copies offsets/tree_of to the device and
 *           allocates the walk buffers of the default launch shape and the
 *           deduplication buffers (about 24 + 4 nb bytes per row plus a sort
 *           workspace of about 12 bytes per row).  It synchronises `stream`.
 * Errors: EINVAL (NULL arrays, mismatched band counts, bad offsets or
 * tree_of, bad nside/theta/flags), EUNSUPPORTED (too many trees, 2^31 rows or
 * more, nside > 16, shared memory exceeded by the deepest tree), ENOMEM,
 * ECUDA.
 */
int trevr2_batch_create(trevr2_tree* const* trees, int ntrees, const int64_t* offsets,
                        const int* tree_of, int nsub, int nside, float theta, uint32_t flags,
                        void* stream, trevr2_batch** out);

/*
 * trevr2_batch_run — enqueues the whole batch: a fixed sequence of kernels
 * (row keys, radix sort, distinct keys, walk, scatter) on `stream`, with no
 * allocation and no synchronisation, so it can be recorded in a CUDA graph.
 *  active  [offsets[nsub]] int64 receiver indices (each in its subset's tree)
 *  J       [offsets[nsub]][nb] float32 output, overwritten
 * Does not synchronise; trevr2_batch_status reports device errors (indices
 * outside [0, N) give NaN rows and EINVAL there).  Runs of one plan must not
 * overlap on the GPU (they share the plan's counter and buffers).
 */
int trevr2_batch_run(trevr2_batch* batch, const int64_t* active, float* J, void* stream);

/*
 * trevr2_batch_autotune — times every launch shape (4 or 8 warps per block,
 * 4 only with TREVR2_BUCKET, x 512, 1024 or 2048 staged sources per warp
 * and pass) on the first
 * min(offsets[nsub], 65536) rows of `active`, keeps the fastest for later
 * runs and re-sizes the buffers for it.  `J` is overwritten (its first rows).
 * warps_out / staging_out (host, may be NULL) receive the chosen shape.
 * Synchronises `stream`.  Errors: EINVAL, ENOMEM, ECUDA.
 */
int trevr2_batch_autotune(trevr2_batch* batch, const int64_t* active, float* J, void* stream,
                          int* warps_out, int* staging_out);

/* Synchronises `stream`; returns (and clears) the device status of the
 * batch's trees (the first error found). */
int trevr2_batch_status(trevr2_batch* batch, void* stream);

/* Releases the plan (not its trees), stream ordered on the last stream used. */
int trevr2_batch_free(trevr2_batch* batch);

/*
 * trevr2_J_batched — one-shot convenience: create, run, status (unless
 * TREVR2_ASYNC, in which case trevr2_status of each tree reports later) and
 * free.  Arguments as for trevr2_batch_create and trevr2_batch_run.
 */
int trevr2_J_batched(trevr2_tree* const* trees, int ntrees, const int64_t* active,
                     const int64_t* offsets, const int* tree_of, int nsub, int nside, float theta,
                     uint32_t flags, float* J, void* stream);

/* Synchronises `stream` and returns (and clears) the tree's device status. */
int trevr2_status(trevr2_tree* tree, void* stream);

/* Releases the tree (stream ordered on the last stream the tree was used on). */
int trevr2_free(trevr2_tree* tree);

/* Message of the last error on the calling thread ("" if none). */
const char* trevr2_last_error(void);

/* ---- Testing aids ---------------------------------------------------
 * These make a later call fail on the host side, so that the error paths of
 * the library can be tested without faulting a GPU.  Process wide, for tests
 * only; both are off by default.
 */
#define TREVR2_DEBUG_FAIL_ALLOC 1   /* value n >= 0: the (n+1)-th device allocation
                                       of the library from now on fails with
                                       ENOMEM (then the setting is off again);
                                       -1 turns it off */
#define TREVR2_DEBUG_SOURCE_STACK 2 /* value c > 0: the warp-wide stack of the
                                       source cut (Sec. 2.5.2) holds at most c
                                       entries, so that a deep cut overflows it
                                       and the walk reports EINTERNAL; 0 restores
                                       the full capacity.  Read when a walk is
                                       set up (trevr2_J, trevr2_J_backward,
                                       trevr2_batch_create) */

/* Sets one testing aid (EINVAL for an unknown `what` or a value out of range). */
int trevr2_debug_set(int what, int64_t value);

/* Bytes the library currently holds in the current device's default
 * stream-ordered memory pool, which only this library allocates from
 * (synchronises the device first; ECUDA if the query fails). */
int trevr2_debug_pool_used(uint64_t* bytes);

/* The architecture the library's kernels run as on the current device
 * (major * 10 + minor of the loaded binary, from the walk kernel's
 * attributes; 103 for sm_103a).  ECUDA without a usable device. */
int trevr2_kernel_binary_version(int* version);

/* Number of CUDA kernels this library has launched in this process so far
 * (a host-side count of launch calls, for accounting in benchmarks). */
uint64_t trevr2_kernel_launches(void);

/* ---- Introspection (tests and tools) --------------------------------- */

typedef struct trevr2_tree_info {
  int64_t n_elements;
  int64_t n_nodes;
  int64_t n_internal;
  int64_t n_leaves;
  int32_t nb;
  int32_t bucket;
  int32_t max_depth;
  int32_t reserved;
  double box_lo[3];
  double box_size;
} trevr2_tree_info;

/* Host copy of the tree's sizes and root cube. */
int trevr2_tree_info_get(const trevr2_tree* tree, trevr2_tree_info* info);

/* Fields for trevr2_tree_export (element fields in sorted order, node fields
 * in node order). */
#define TREVR2_F_KEYS 1        /* uint64 [N] sorted Morton keys                  */
#define TREVR2_F_PERM 2        /* int32  [N] sorted position -> caller index     */
#define TREVR2_F_PREFIX 3      /* uint64 [n] node key prefix                     */
#define TREVR2_F_DEPTH 4       /* int32  [n] node depth                          */
#define TREVR2_F_FIRST 5       /* int32  [n] first element (sorted position)     */
#define TREVR2_F_COUNT 6       /* int32  [n] element count                       */
#define TREVR2_F_CHILD 7       /* int32  [n] lower child (upper = +1), -1 leaf   */
#define TREVR2_F_PARENT 8      /* int32  [n] parent, -1 for the root             */
#define TREVR2_F_LUM 9         /* float32 [n][nb] summed luminosity             */
#define TREVR2_F_CENTRE 10     /* float64 [n][3] centre of luminosity (caller units) */
#define TREVR2_F_ALPHA_LEAF 11 /* float32 [n][nb] bucket absorption (caller units), 0 internal */
#define TREVR2_F_B 12          /* float64 [n] largest centre-to-corner distance (caller units) */

/* Copies one field into `dst` (device, at least `bytes` bytes). */
int trevr2_tree_export(const trevr2_tree* tree, int field, void* dst, size_t bytes, void* stream);

/* Per-direction absorption of every node for one nside, as float32
 * [n_nodes][6 nside^2][nb] in caller units (leaves repeat their isotropic
 * value); builds and caches the tables if needed. */
int trevr2_alpha_table(trevr2_tree* tree, int nside, float* dst, size_t bytes, void* stream);

/* HEALPix RING pixel centres, float64 [12 nside^2][3] (Gorski et al. 2005). */
int trevr2_healpix_pix2vec(int nside, double* dst, void* stream);

/* HEALPix RING pixel of each of n direction vectors (float64 [n][3]),
 * int32 [n] (Gorski et al. 2005). */
int trevr2_healpix_vec2pix(int nside, const double* v, int64_t n, int32_t* pix, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* TREVR2_H */
