/*
 * nl.h -- C ABI of the GB300 (sm_103a) compressed cluster neighbor list.
 *
 * Method: "GPU-Native Compressed Neighbor Lists with a Space-Filling-Curve
 * Data Layout" (Thaler & Keller), Sec. II.  The library builds, on one GPU,
 * the paper's neighbor list over SFC-sorted particles with per-particle
 * interaction radii, and runs neighborhood passes that decode it:
 *
 *   SFC keys -> stable radix sort -> clusters of M consecutive particles and
 *   super-clusters of 8 clusters (Sec. II-A) -> octree from the sorted keys
 *   (Sec. II-A) -> cluster-pair search against bounding boxes inflated by the
 *   largest radius -> one record per super-cluster: count, 8-bit masks, and
 *   the nibble-compressed j-cluster indices (Sec. II-A/B/C) -> decode inside
 *   the SPH density / force, Lennard-Jones (+ Coulomb), neighbor-count and
 *   nearest-neighbor passes (Sec. II-A, II-D).  Lists are stored in full or
 *   with every pair of clusters of two super-clusters once (half lists,
 *   Sec. II-D), and can take new positions for several steps (Sec. III-B).
 *
 * Conventions shared by every entry point:
 *  - Particle arrays are DEVICE pointers in the caller's order, borrowed for
 *    the duration of the call (nl_build copies what it keeps).  Outputs are
 *    written in caller order.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Work is
 *    enqueued on it; calls that must read a device word back synchronise that
 *    stream and say so.
 *  - No exception crosses the ABI.  Every call returns an nl_status; on any
 *    status other than NL_OK, nl_last_error() (thread-local) describes it and
 *    no output array of that call is guaranteed to have been written.
 *  - The pair predicate is fixed in IEEE FP32 without FMA contraction:
 *      dx = xj - xi, wrapped once by +-L on a periodic axis when |dx| > L/2,
 *      d2 = (dx*dx + dy*dy) + dz*dz, r = support*h,
 *      symmetric pair (the list): i != j and d2 < max(ri, rj)^2
 *      gather pair (density, counts, LJ, nearest): i != j and d2 < ri^2.
 */
#ifndef NL_H
#define NL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    NL_OK = 0,
    NL_ERR_ARG = 1,            /* bad argument: NULL pointer, n < 1, non-finite or
                                  out-of-box coordinate, h <= 0 or non-finite */
    NL_ERR_RADIUS = 2,         /* support * max(h) >= L/2 on a periodic axis */
    NL_ERR_OOM = 3,            /* device allocation failed (no partial state kept) */
    NL_ERR_CUDA = 4,           /* a CUDA runtime call failed */
    NL_ERR_CAPACITY = 5,       /* a bounded buffer overflowed and could not grow */
    NL_ERR_NOT_CONVERGED = 6,  /* h iteration hit its iteration cap */
    NL_ERR_TIMEOUT = 7,        /* a bounded device loop gave up */
    NL_ERR_UNIMPLEMENTED = 8
} nl_status;

enum { NL_KEY_MORTON = 0, NL_KEY_HILBERT = 1 };

/* Simulation box.  Every coordinate must satisfy lo <= x <= hi on every
 * axis; periodic[a] != 0 makes axis a periodic with length L = hi - lo
 * (computed in FP32).  Sec. II-A: periodic distances are always computed,
 * no shift vectors are stored. */
typedef struct {
    float lo[3];
    float hi[3];
    int32_t periodic[3];
} nl_box;

/* Build options (Sec. II-D: cluster and super-cluster sizes, compression). */
typedef struct {
    int32_t key;          /* NL_KEY_MORTON or NL_KEY_HILBERT (63-bit keys, 21 bits/axis) */
    int32_t cluster;      /* particles per i-cluster M: 4, 8 or 16; super-cluster = 8 i-clusters */
    float support;        /* interaction radius r_i = support * h_i (2 for the cubic spline) */
    int32_t compress;     /* 1: nibble codec (Sec. II-B); 0: raw u32 cluster indices */
    int32_t leaf_bucket;  /* octree leaf capacity B in particles, 8..1024 (default 256) */
    int32_t threads_per_block; /* search / pass block shape: 128 or 256 threads (0 = 256) */
    int32_t blocks_per_sm;     /* persistent grids: blocks per SM, 1..8 (0 = 3 search, 4 pass) */
    int32_t j_cluster;    /* particles per j-cluster MJ: 0 (= M), M, or M / 2 when M >= 8;
                             the M x MJ tiles of Sec. II-A / III-A (8 x 4 is the paper's
                             NVIDIA choice).  Stored list indices count j-clusters. */
    int32_t half_list;    /* 1: store every cluster pair once (the symmetric list of
                             Sec. II-D): the record of super-cluster s holds only the
                             j-clusters J >= 8s of its full record, with the same masks,
                             and every pass adds each pair to both of its particles
                             (density and counts as integers: the same bits on every
                             run; forces as FP64 sums rounded once to FP32, where the
                             order of the adds can move the last bit in rare ties).
                             Needs MJ = M.  The h iteration always builds full lists. */
} nl_params;

/* Fills p with {NL_KEY_HILBERT, 8, 2.0f, 1, 256, 0, 0, 0, 0}. */
void nl_default_params(nl_params *p);

typedef struct nl_list nl_list; /* opaque; owns all of its device memory */

/* Sizes and statistics of a built list (host struct). */
typedef struct {
    int64_t n;               /* particles */
    int64_t n_clusters;      /* ceil(n / M) rounded up to whole super-clusters */
    int64_t n_superclusters; /* clusters / 8 */
    int64_t n_leaves;        /* octree leaves (non-empty cells) */
    int64_t n_nodes;         /* octree nodes, pre-order */
    int64_t n_entries;       /* stored (j-cluster, mask) entries */
    int64_t n_tiles;         /* sum over entries of popcount(mask): computed cluster pairs */
    int64_t list_bytes;      /* bytes of all super-cluster records */
    int32_t cluster;         /* M */
    int32_t compress;
    /* work of the last cluster-pair search (all rounds) */
    int64_t node_visits;     /* octree nodes tested, summed over super-clusters */
    int64_t leaf_visits;     /* leaves reached */
    int64_t j_examined;      /* j-clusters box-tested against a super-cluster */
    int64_t tile_tests;      /* (i-cluster, j-cluster) tiles decided by the exact predicate */
    int32_t j_cluster;       /* MJ */
    int32_t pad0;
} nl_sizes;

/* Builds a new list (Sec. II-A, Listing "build"): keys, sort, clusters,
 * octree, cluster-pair search, encoding.  x,y,z,h: n device floats (caller
 * order).  On success *out owns the list; on failure *out is NULL.
 * Synchronises `stream` twice (validation + size word, final status).
 * NL_ERR_TIMEOUT if a tile of the key sort waited in vain (a bounded wait)
 * for the counts of the tiles before it; nothing of the list is kept. */
nl_status nl_build(const float *x, const float *y, const float *z, const float *h, int64_t n,
                   const nl_box *box, const nl_params *p, void *stream, nl_list **out);

/* Same as nl_build into an existing list, reusing its device buffers (they
 * only grow).  On failure the list is left empty (n = 0) but valid. */
nl_status nl_rebuild(nl_list *nl, const float *x, const float *y, const float *z, const float *h,
                     int64_t n, const nl_box *box, const nl_params *p, void *stream);

/* SPH density (Sec. II-D): rho_i = m_i W(0,h_i) + sum_{j gather pair} m_j W(r_ij,h_i),
 * W the M4 cubic spline with support 2h: W = w(r/h)/(pi h^3),
 * w = 1 - 1.5q^2 + 0.75q^3 (q<1), 0.25(2-q)^3 (1<=q<2), 0 beyond.
 * m: n device floats (caller order); rho: n device floats written in caller
 * order.  FP32 arithmetic.  Does not synchronise. */
nl_status nl_density_pass(const nl_list *nl, const float *m, float *rho, void *stream);

/* Force passes over the list (Sec. II-D pair functions; Sec. III-B LJ).
 *  NL_FORCE_SPH_PRESSURE: over symmetric pairs (i != j, d2 < max(ri,rj)^2),
 *    a_i = -sum_j m_j [P_i/rho_i^2 grad_i W(r_ij,h_i) + P_j/rho_j^2 grad_i W(r_ij,h_j)],
 *    grad_i W(r,h) = w'(r/h) / (pi h^4) * (x_i - x_j) / r, W the cubic spline of
 *    nl_density_pass.  m, rho, pres: n device floats (caller order); params unused.
 *  NL_FORCE_LJ: over gather pairs (i != j, d2 < ri^2),
 *    F_i = sum_j 24 eps (2 sigma^12 / r^14 - sigma^6 / r^8) (x_i - x_j);
 *    params = host {eps, sigma}; m, rho, pres unused (may be NULL).
 *  NL_FORCE_LJ_COULOMB (Sec. III-B: 12/6 Lennard-Jones and Coulomb, the list
 *    built at a larger radius than the interaction cutoff): over the listed
 *    gather pairs inside the cutoff (i != j, d2 < ri^2 and d2 < rc^2, rc^2
 *    rounded once in FP32),
 *    F_i = sum_j [24 eps (2 sigma^12 / r^14 - sigma^6 / r^8) + kc q_i q_j / r^3] (x_i - x_j),
 *    plain cutoff (no shift).  params = host {eps, sigma, rc, kc}, rc = 0 for
 *    the list radius alone; m = the charges q (n device floats, caller order;
 *    NULL: all zero); rho, pres unused.  NL_ERR_ARG for non-finite eps, kc or
 *    rc, sigma <= 0 or rc < 0.  With rc below every list radius the result is
 *    the force over all pairs within rc, also after nl_refresh_positions as
 *    long as twice its max_disp stays below min(ri) - rc.
 * ax, ay, az: n device floats written in caller order.  FP32 arithmetic with
 * block-partial sums; on a half list each pair also gives particle j its
 * force (SPH: -m_i/m_j times i's pair term; LJ, LJ + Coulomb: -F_ij when
 * d2 < rj^2), the shares summed in FP64.  Does not synchronise. */
enum { NL_FORCE_SPH_PRESSURE = 0, NL_FORCE_LJ = 1, NL_FORCE_LJ_COULOMB = 2 };
nl_status nl_force_pass(const nl_list *nl, int32_t kind, const float *params, const float *m,
                        const float *rho, const float *pres, float *ax, float *ay, float *az,
                        void *stream);

/* Gather-neighbor count of every particle (j != i with d2 < ri^2), caller
 * order, n device uint32.  Does not synchronise. */
nl_status nl_neighbor_counts(const nl_list *nl, uint32_t *counts, void *stream);

/* Distance from every particle to its nearest gather neighbor (j != i with
 * d2 < ri^2): the pair function of Sec. II-D with a minimum reduction.  dist:
 * n device floats, caller order; +inf for a particle without a neighbor.
 * FP32 sqrt of the smallest squared distance (the accurate wrapped difference
 * on periodic axes).  A minimum does not depend on the order of its
 * operands, so full and half lists give the same bits.  Does not synchronise. */
nl_status nl_nearest_distance(const nl_list *nl, float *dist, void *stream);

/* List reuse across steps (the Verlet buffer of Sec. III-B and its
 * production remark: a list built at radius r_list serves an interaction
 * cutoff rc < r_list while particles move less than (r_list - rc)/2).
 * x, y, z: n device floats in caller order, the new positions, on periodic
 * axes inside [lo, hi) as for nl_build; h and the list are kept.  The passes
 * that follow read these positions and the listed pairs; on periodic systems
 * the super-clusters that may hold a wrapped pair are found again for the new
 * positions (two small kernels), so the others keep the kernel without
 * periodic arithmetic.  max_disp: one
 * device float or NULL; set to the largest displacement of any particle from
 * the positions the list was built on (minimum image on periodic axes, FP32),
 * so that the caller rebuilds once 2 * max_disp reaches r_list - rc.  The
 * next build or rebuild drops the reference positions.  NL_ERR_ARG for an
 * empty list or a NULL array.  Does not synchronise. */
nl_status nl_refresh_positions(nl_list *nl, const float *x, const float *y, const float *z,
                               float *max_disp, void *stream);

/* Releases the list and its device memory (after the stream work using it
 * has completed; nl_free synchronises the device).  nl_free(NULL) = NL_OK. */
nl_status nl_free(nl_list *nl);

/* Host copy of the list sizes and statistics. */
nl_status nl_get_sizes(const nl_list *nl, nl_sizes *out);

/* Inspection copies to HOST buffers (tests, tools); each synchronises.
 * keys: n uint64 sorted SFC keys; perm: n int32, perm[k] = caller index of
 * the particle at sorted position k. */
nl_status nl_copy_sorted(const nl_list *nl, uint64_t *keys, int32_t *perm);

/* Octree in pre-order, n_nodes entries each: level, first and end particle
 * (sorted positions, end exclusive), leaf flag, skip (index of the next node
 * after this node's subtree). */
nl_status nl_copy_octree(const nl_list *nl, int32_t *level, int32_t *first, int32_t *end,
                         int32_t *leaf, int32_t *skip);

/* Records: rec_off[s] = byte offset of super-cluster s's record inside the
 * list buffer (n_superclusters entries); bytes: list_bytes bytes.  Record
 * layout: u32 count | count u8 masks, zero-padded to 4 bytes | nibble stream
 * (compressed) or count u32 (raw), zero-padded to 4 bytes.  The stream holds
 * blocks of 32 index differences (d0 = J0 + 1, dk = Jk - J(k-1)): a 32-bit
 * mask (bit k set iff dk != 1), one info nibble per set bit (dk+6 for dk in
 * [2,9], else the value's nibble count minus one), then the data nibbles of
 * every dk >= 10, most significant first; nibble p is byte p/2, low half for
 * even p (Sec. II-B Tables 1-2, Sec. II-C). */
nl_status nl_copy_records(const nl_list *nl, uint64_t *rec_off, uint8_t *bytes);

/* End-to-end convenience call on HOST buffers: copies x, y, z, h, m (n
 * floats each, pageable or pinned host memory) into device buffers owned by
 * the list (z and h on a second stream of the list beside x and y, m on a
 * third while the list is built),
 * rebuilds the list (as nl_rebuild), runs nl_density_pass and copies rho
 * (n floats) back to host memory.  Synchronises `stream`. */
nl_status nl_density_from_host(nl_list *nl, const float *x, const float *y, const float *z,
                               const float *h, const float *m, int64_t n, const nl_box *box,
                               const nl_params *p, float *rho, void *stream);

/* Stage timing.  When enabled on a list, the build and the passes record
 * CUDA events on their stream around each stage; nl_get_stage_times writes
 * the durations in milliseconds of the most recent build / pass to ms[0..):
 * 0 keys+validation, 1 radix sort, 2 permute+cluster boxes, 3 octree,
 * 4 cluster-pair search (+ encoding in the full search), 5 record assembly
 * of the half search (tuple sort, scan, encoding; 0 for the full search),
 * 6 pass input gather, 7 pass kernel.
 * *count receives the number of stages (8).  Synchronises the device. */
nl_status nl_set_profiling(nl_list *nl, int32_t on);
nl_status nl_get_stage_times(const nl_list *nl, float *ms, int32_t cap, int32_t *count);

/* Creates an empty list handle (no device memory yet) for nl_rebuild or
 * nl_density_from_host. */
nl_status nl_create(nl_list **out);

/* Smoothing-length iteration (not in the paper; the workloads need
 * per-particle h at a target neighbor count).  Finds for every particle an h
 * with |#{j != i : d2 < (support*h)^2} - n_target| <= tol, counting with the
 * canonical FP32 distance.  Counts come from neighbor lists built at search
 * radius (1 + margin) * support * h; a list is rebuilt only when an h
 * outgrows it.  Update per particle: bracket the window, step
 * h * (n_target / count)^(1/3) clamped to [1/2, 2] while one side is open,
 * then bisect the bracket in h^3.
 *   start = NL_HSTART_GIVEN: h (device, caller order) holds the initial guess;
 *   start = NL_HSTART_PLAIN: the initial guess is computed per super-cluster
 *           from its bounding-box volume, h = 0.5 (3 n_target V / (4 pi count))^(1/3),
 *           and h's input values are ignored.
 * On return h holds the iterated values (caller order) and, if converged is
 * not NULL, converged[i] (device, caller order) is 1 for particles inside the
 * window.  Returns NL_ERR_NOT_CONVERGED when max_iter passes leave particles
 * outside (h and flags are still written).  The list is left built at the
 * search radius: rebuild with the returned h before running passes.
 * Synchronises `stream` once per iteration. */
enum { NL_HSTART_GIVEN = 0, NL_HSTART_PLAIN = 1 };
typedef struct {
    int32_t iterations;   /* count passes run */
    int32_t rebuilds;     /* list searches run */
    int64_t unconverged;  /* particles outside the window at return */
} nl_hiter_info;
nl_status nl_iterate_h(nl_list *nl, const float *x, const float *y, const float *z, float *h,
                       int64_t n, const nl_box *box, const nl_params *p, float n_target, float tol,
                       int32_t max_iter, float margin, int32_t start, uint8_t *converged,
                       nl_hiter_info *info, void *stream);

/* Per-pass record of the last nl_iterate_h / nl_iterate_h_batch on this
 * list: whether the pass rebuilt the list first, the super-clusters it
 * counted (all on the first pass, then the ones with unconverged particles),
 * the particles still outside the window after it, the list's entries and
 * computed cluster pairs (tiles) at that pass, and its host wall time in ms
 * (every pass ends with a stream synchronisation).  Copies
 * min(cap, passes) records; *count = passes. */
typedef struct {
    int32_t rebuilt;
    int32_t pad0;
    int64_t active;
    int64_t unconverged;
    int64_t entries;
    int64_t tiles;
    float ms;
    int32_t pad1;
} nl_hiter_step;
nl_status nl_get_hiter_trace(const nl_list *nl, nl_hiter_step *steps, int32_t cap, int32_t *count);

/* Allocation-free SFC ordering.  The paper has no counterpart: this entry
 * point exists for callers that cannot allocate device memory where they
 * need the order: a latency-critical simulation loop that cannot afford
 * cudaMalloc's implicit device synchronisation, or a host framework that owns
 * all device memory through its own pool and forbids driver allocations by
 * the libraries it calls.  It computes exactly what nl_build
 * computes for its first two steps: keys[k] = the k-th smallest 63-bit SFC
 * key (NL_KEY_MORTON or NL_KEY_HILBERT) and perm[k] = the caller index of
 * that particle (stable: equal keys keep caller order), for n <= 1048576.
 * x, y, z, h: n device floats (caller order), validated as in nl_build;
 * keys (n uint64) and perm (n uint32) are device arrays owned by the caller.
 * Scratch comes from a fixed device array inside the library (about
 * 14.7 MB, held by every GPU that loads the library until exit); nothing is
 * allocated.  The first call made with a device current looks up that
 * array's address on that device (cudaGetSymbolAddress); make that first call
 * before any stream capture begins.  Concurrent calls that overlap on
 * the GPU share the array and race; serialise them.  n > NL_NOALLOC_MAX_N
 * returns NL_ERR_ARG.  Synchronises `stream` (one status read). */
#define NL_NOALLOC_MAX_N 1048576
nl_status nl_sfc_order_noalloc(const float *x, const float *y, const float *z, const float *h,
                               int64_t n, const nl_box *box, int32_t key, float support,
                               uint64_t *keys, uint32_t *perm, void *stream);

/* Batches of independent systems (the workloads' "many uneven systems").
 * The caller's arrays hold nsys systems back to back: system s owns
 * indices [offsets[s], offsets[s+1]) (host int64 array of nsys+1 entries,
 * offsets[0] = 0, every system non-empty) and has its own box boxes[s]
 * (host array).  Every stage runs once for the whole batch: one key kernel,
 * one radix sort ordering (system, key), one permutation that starts every
 * system on a super-cluster boundary, one octree pass producing each
 * system's pre-order octree, one persistent search launch and one
 * persistent pass launch over all super-clusters.  Pairs never cross
 * systems; results equal those of building every system on its own (the
 * records hold batch-global cluster indices).  Passes, counts, forces and
 * inspection calls accept batched lists unchanged (caller order). */
nl_status nl_build_batch(const float *x, const float *y, const float *z, const float *h,
                         int32_t nsys, const int64_t *offsets, const nl_box *boxes,
                         const nl_params *p, void *stream, nl_list **out);
nl_status nl_rebuild_batch(nl_list *nl, const float *x, const float *y, const float *z,
                           const float *h, int32_t nsys, const int64_t *offsets,
                           const nl_box *boxes, const nl_params *p, void *stream);
nl_status nl_iterate_h_batch(nl_list *nl, const float *x, const float *y, const float *z, float *h,
                             int32_t nsys, const int64_t *offsets, const nl_box *boxes,
                             const nl_params *p, float n_target, float tol, int32_t max_iter,
                             float margin, int32_t start, uint8_t *converged, nl_hiter_info *info,
                             void *stream);

/* One step of a batch (build + density pass) as a CUDA graph.  The list is
 * first built normally (buffers sized with slack, inputs validated), then
 * the sync-free form of the same step -- keys, radix sort, permutation,
 * octree with device-side counts, one persistent search launch, input
 * gather and one persistent density launch -- is captured on `stream` and
 * instantiated.  nl_graph_launch replays it; the device arrays x, y, z, h,
 * m, rho must stay allocated at the same addresses (their contents may
 * change between launches).  A replay never allocates or synchronises, so
 * capacity overflows (more octree nodes or longer lists than the slack
 * allows) and invalid inputs are only recorded on the device:
 * nl_graph_check synchronises `stream` and returns NL_ERR_CAPACITY,
 * NL_ERR_ARG or NL_ERR_RADIUS for the last replay (then rebuild without the
 * graph and create a new one), else NL_OK and refreshes nl_get_sizes. */
typedef struct nl_graph nl_graph;
nl_status nl_graph_create(nl_list *nl, const float *x, const float *y, const float *z,
                          const float *h, const float *m, float *rho, int32_t nsys,
                          const int64_t *offsets, const nl_box *boxes, const nl_params *p,
                          void *stream, nl_graph **out);
nl_status nl_graph_launch(nl_graph *g, void *stream);
nl_status nl_graph_check(nl_graph *g, void *stream);
nl_status nl_graph_free(nl_graph *g);

/* Autotuner: times build + density of the given batch for every candidate
 * tile shape M x MJ in {4x4, 8x8, 8x4, 16x16, 16x8}, block shape in {128, 256} threads and
 * persistent-grid occupancy in {2, 3, 4} blocks per SM (reps timed runs
 * each after one warm-up, CUDA events on `stream`; with base->half_list only
 * the shapes with MJ = M) and writes the fastest
 * parameters (other fields copied from *base) to *best and its mean time
 * to *best_ms.  Synchronises `stream`. */
nl_status nl_autotune_batch(const float *x, const float *y, const float *z, const float *h,
                            const float *m, int32_t nsys, const int64_t *offsets,
                            const nl_box *boxes, const nl_params *base, int32_t reps,
                            nl_params *best, float *best_ms, void *stream);

/* Learned start for the h iteration (not in the paper).  A small MLP maps
 * per-cluster SFC density features to log(h / e64) (e64 = largest side of
 * the cluster's super-cluster box): 8 features -> 64 -> 64 -> 64 (SiLU) -> 1,
 * BF16 tensor-core matrix products with FP32 accumulation, FP32 master
 * weights, Adam.  Features of cluster c, with e(B) the largest side of box B,
 * e8 the cluster box, e512 / e4096 the boxes of the 8 / 64 super-clusters
 * around it in its system, L the largest side of the system box and N_s its
 * particle count: log(e8/e64), log(e512/e64), log(e4096/e64), log(ex/e8),
 * log(ey/e8), log(ez/e8), log(count/M), log(e64/L) + log(N_s)/3.
 * Parameters are packed W1 (64x8, row-major out x in) b1 W2 (64x64) b2
 * W3 (64x64) b3 W4 (64) b4: nl_mlp_nparams() floats. */
typedef struct nl_mlp nl_mlp;
int64_t nl_mlp_nparams(void);
/* Random initialisation (normal, std 1/sqrt(fan-in); zero biases). */
nl_status nl_mlp_create(uint64_t seed, nl_mlp **out);
nl_status nl_mlp_free(nl_mlp *mlp);
/* Host copies of the FP32 parameters (checkpoints). */
nl_status nl_mlp_get_params(const nl_mlp *mlp, float *params);
nl_status nl_mlp_set_params(nl_mlp *mlp, const float *params);
/* Features X (n_clusters x 8, device) and e64 (n_superclusters, device) of a
 * built list (any smoothing lengths: features depend on positions only). */
nl_status nl_mlp_features(const nl_list *nl, float *X, float *e64, void *stream);
/* Training targets of a built list from converged h (device, caller order):
 * y[c] = log(mean h over the real particles of cluster c / e64), w[c] = 1,
 * and y = w = 0 for clusters without real particles. */
nl_status nl_mlp_targets(const nl_list *nl, const float *h, const float *e64, float *y, float *w,
                         void *stream);
/* Gradient (device, nl_mlp_nparams floats) and value (*loss, host) of
 * (1/n) sum_r w_r (pred_r - y_r)^2 over n samples; synchronises. */
nl_status nl_mlp_grad(nl_mlp *mlp, const float *X, const float *y, const float *w, int64_t n,
                      float *grad, float *loss, void *stream);
/* Minibatch Adam training for `epochs` passes over n samples (shuffled with
 * `seed`); *loss receives the mean loss of the last epoch.  Synchronises. */
nl_status nl_mlp_train(nl_mlp *mlp, const float *X, const float *y, const float *w, int64_t n,
                       int32_t epochs, int32_t batch, float lr, uint64_t seed, float *loss,
                       void *stream);
nl_status nl_mlp_predict(const nl_mlp *mlp, const float *X, int64_t n, float *pred, void *stream);
/* Attaches a model to a list; nl_iterate_h(_batch) with start =
 * NL_HSTART_LEARNED then starts every particle at e64 * exp(prediction of
 * its cluster).  The exact iteration still decides the result. */
enum { NL_HSTART_LEARNED = 2 };
nl_status nl_set_mlp(nl_list *nl, const nl_mlp *mlp);

/* Thread-local description of the last error (never NULL). */
const char *nl_last_error(void);

/* SFC domain decomposition across ranks (Sec. I: the domain is split into
 * contiguous key ranges of the space-filling curve; Sec. IV: every rank builds
 * its list over its own particles plus a halo received from the others).
 * These are the per-rank device steps; the caller exchanges their results
 * between ranks (paper_2602_19873_gb300/domain.py does it over
 * torch.distributed: two all-reduces of key histograms for the splitters,
 * one all-to-all of the particles, one all-gather of the rank boxes, one
 * all-to-all of the halo).  At most 64 ranks: destinations are the bits of a
 * 64-bit mask per particle.  All arrays are device arrays in the caller's
 * order; none of these calls synchronises except nl_sfc_keys.
 *
 * nl_sfc_keys: the 63-bit key of every particle in `box` exactly as nl_build
 *   computes it (NL_KEY_MORTON / NL_KEY_HILBERT, 21 bits per axis), caller
 *   order, unsorted.  Validates like nl_build (NL_ERR_ARG, NL_ERR_RADIUS);
 *   allocates stream-ordered scratch (4n + 256 bytes) and synchronises
 *   `stream` once.  n = 0 is allowed (nothing written). */
nl_status nl_sfc_keys(const float *x, const float *y, const float *z, const float *h, int64_t n,
                      const nl_box *box, int32_t key, float support, uint64_t *keys, void *stream);
/* hist[b] = #{i : keys[i] >= lo and (keys[i] - lo) >> shift == b}, b < nbins
 *   (nbins uint64 counters, overwritten).  0 <= shift <= 63, 1 <= nbins <= 2^24. */
nl_status nl_key_histogram(const uint64_t *keys, int64_t n, uint64_t lo, int32_t shift,
                           int32_t nbins, uint64_t *hist, void *stream);
/* mask[i] = 1 << (number of splitters <= keys[i]): the owner rank of every
 *   particle, for P ranks and P-1 ascending splitters (device uint64). */
nl_status nl_domain_owner_mask(const uint64_t *keys, int64_t n, const uint64_t *splitters,
                               int32_t P, uint64_t *mask, void *stream);
/* out[0..7] = lo.x lo.y lo.z rmax hi.x hi.y hi.z 0: the tight box of the
 *   particles and their largest radius support*h (device floats; n = 0 gives
 *   lo = +inf, hi = -inf, rmax = 0).  Allocates 32 bytes stream-ordered. */
nl_status nl_domain_box(const float *x, const float *y, const float *z, const float *h,
                        int64_t n, float support, float *out, void *stream);
/* Halo destinations: mask[i] bit q (q != self) is set when particle i, of
 *   radius support*h_i, could be a symmetric neighbor of some particle inside
 *   rank q's box dom[8q .. 8q+7] (the layout of nl_domain_box; an empty box
 *   is skipped): the search's conservative point-box test with monotone
 *   rounding and periodic gaps of `box`, so no pair of the predicate is lost.
 *   dom: P x 8 device floats, 16-byte aligned. */
nl_status nl_domain_halo_mask(const float *x, const float *y, const float *z, const float *h,
                              int64_t n, const nl_box *box, float support, const float *dom,
                              int32_t P, int32_t self, uint64_t *mask, void *stream);
/* counts[q] = number of set bits q over the n masks (P device int64). */
nl_status nl_domain_count(const uint64_t *mask, int64_t n, int32_t P, int64_t *counts,
                          void *stream);
/* Stable grouping by destination: for every bit q of mask[i], i is written to
 *   idx[offsets[q] + (number of j < i with bit q)].  offsets: P device int64
 *   (typically the exclusive sums of nl_domain_count); idx must hold every
 *   destination's range.  n <= 2^32.  Allocates 4 P ceil(n/1024) bytes
 *   stream-ordered. */
nl_status nl_domain_group(const uint64_t *mask, int64_t n, int32_t P, const int64_t *offsets,
                          uint32_t *idx, void *stream);

/* Measured FP32 rate of the current GPU, the denominator of the rooflines of
 * the search and the passes (bound by FP32 issue, not memory).  The paper has
 * no counterpart; it is measurement support.  Runs independent fused
 * multiply-add chains on every lane of every SM -- scalar fma.rn.f32
 * (packed = 0) or the two-element fma.rn.f32x2 (packed = 1) -- and times
 * reps launches (after one warm-up) with CUDA events on `stream`.
 * *ops_per_s = FP32 element operations per second of the fastest launch (one
 * add, multiply, fused multiply-add or compare of one element = one op; a
 * packed instruction = two); *ms_out (may be NULL) = that launch's time.
 * reps in 1..1000, else NL_ERR_ARG.  Allocates one word (stream-ordered) and
 * synchronises `stream` once per launch. */
nl_status nl_probe_fp32_rate(int32_t packed, int32_t reps, double *ops_per_s, double *ms_out,
                             void *stream);

#ifdef __cplusplus
}
#endif
#endif /* NL_H */
