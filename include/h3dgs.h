/*
 * h3dgs.h -- C ABI of the B300 (sm_103a) hierarchical 3D Gaussian render path.
 *
 * Method: "A Hierarchical 3D Gaussian Representation for Real-Time Rendering of Very Large
 * Datasets" (Kerbl, Meuleman, Kopanas, Wimmer, Lanvin, Drettakis; ACM TOG 43(4), 2024).
 *
 * Per view, the library selects a cut through a Gaussian hierarchy at a target granularity tau
 * (Sec. 4.2), interpolates each cut node with its parent (Sec. 4.2, Eq. t_interp and
 * Eq. alphap), and splats the result with a tile-based rasteriser (Sec. 3.1, Eq. alpha;
 * EWA low-pass of Sec. 5.1).  It also provides the adjoint used to optimise interior nodes
 * (Sec. 5.1, Sec. 7.1, Sec. 7.3).
 *
 * Conventions shared by every call
 *   - All attribute, topology, output and gradient buffers are DEVICE pointers unless a
 *     parameter says "host".  The caller owns them; the library never frees them.
 *   - Every call is asynchronous on the stream given to h3dgs_create, unless stated otherwise.
 *     Results are valid once that stream has synchronised.
 *   - Every call returns an h3dgs_status and never aborts, traps or prints.  On failure,
 *     h3dgs_last_error() returns a one-line message.  A context is NOT thread-safe.
 *   - Floating point is fp32 throughout.  Integer decisions (cut membership, tile rectangles,
 *     depth order) are evaluated in a fixed fp32 operation order documented with each call.
 */
#ifndef H3DGS_H
#define H3DGS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    H3DGS_OK = 0,
    H3DGS_ERR_INVALID_ARG = 1, /* null pointer, bad size or alignment, n_cams out of range    */
    H3DGS_ERR_OOM = 2,         /* workspace allocation failed                                  */
    H3DGS_ERR_CUDA = 3,        /* a CUDA runtime call failed (message has the CUDA error)      */
    H3DGS_ERR_CAPACITY = 4,    /* an output or a fixed workspace was too small (see each call) */
    H3DGS_ERR_TIMEOUT = 5,     /* a bounded device-side wait gave up                           */
    H3DGS_ERR_STATE = 6,       /* call order violated (no hierarchy, no saved forward state)   */
    H3DGS_ERR_NO_DEVICE = 7    /* no CUDA device, or the device is not sm_103                  */
} h3dgs_status;

typedef struct h3dgs_ctx h3dgs_ctx; /* opaque */

/* Pinhole camera.  World -> camera: x_c = R x_w + T, R row-major; camera axes x right, y down,
 * z forward.  Pixel (i, j) covers [i, i+1) x [j, j+1) and is sampled at (i + 0.5, j + 0.5):
 * u = fx x_c/z_c + cx, v = fy y_c/z_c + cy.  Points with z_c <= znear are culled.  tau is the
 * target granularity in pixels (Sec. 4.2). */
typedef struct {
    float R[9];
    float T[3];
    float fx, fy, cx, cy;
    int32_t width, height;
    float znear;
    float tau;
} h3dgs_camera;

/* A Gaussian hierarchy (Sec. 4.1) as device arrays, one row per node, in breadth-first order:
 * node 0 is the root (parent[0] = -1), the children of a node are contiguous
 * (child_start .. child_start + child_count - 1), parent < child, leaves have child_count 0.
 * Attributes are ACTIVATED values: scale > 0 (metres), rot a quaternion (w, x, y, z) (need not
 * be unit length), opacity >= 0 (interior nodes carry the falloff of Sec. 4.1, which may exceed
 * 1), sh the 16 degree-3 SH coefficients per colour channel laid out [k*3 + channel].
 * box_min/box_max: the AABB of the 3-sigma boxes of all leaves below the node (Sec. 4.2); every
 * parent box must contain its children's boxes.
 * Alignment: every pointer 16-byte aligned (rot and sh rows are read as float4). */
typedef struct {
    int64_t n_nodes;
    const float* mean;          /* [N,3]  */
    const float* scale;         /* [N,3]  */
    const float* rot;           /* [N,4]  */
    const float* opacity;       /* [N]    */
    const float* sh;            /* [N,48] */
    const float* box_min;       /* [N,3]  */
    const float* box_max;       /* [N,3]  */
    const int32_t* parent;      /* [N]    */
    const int32_t* child_start; /* [N]    */
    const int32_t* child_count; /* [N]    */
} h3dgs_hierarchy;

/* Gradients of the node attributes, same layouts as h3dgs_hierarchy (device, accumulated +=). */
typedef struct {
    float* mean;    /* [N,3]  */
    float* scale;   /* [N,3]  */
    float* rot;     /* [N,4]  */
    float* opacity; /* [N]    */
    float* sh;      /* [N,48] */
} h3dgs_grads;

/* Render options.  h3dgs_default_opts() fills the values used by the paper and by 3DGS. */
typedef struct {
    int32_t tile_w, tile_h;  /* screen tile in pixels: 16x16 (default), 8x8, 32x8, 8x32 or 16x8
                                (both sides multiples of 8: a warp blends 8x8 pixels)          */
    float lowpass;           /* screen-space variance added to the 2D covariance, px^2 (0.3)    */
    float alpha_clamp;       /* alpha upper clamp (0.99, Sec. 7.3)                              */
    float alpha_floor;       /* alpha below which a splat is skipped (1/255)                   */
    float t_min;             /* stop before transmittance would drop below this (1e-4)        */
    int32_t aa_compensate;   /* 1: opacities scaled by sqrt(det S' / det(S' + lowpass I))     */
    int32_t interpolate;     /* 1: parent/child interpolation (Sec. 4.2); 0: render the cut as is */
    float bg[3];             /* background colour                                              */
    int32_t blend_chunk;     /* a tile list of L > blend_chunk entries is blended as
                                ceil(L / blend_chunk) chunks of near-equal length by separate
                                CTAs (64 .. 65536); 0 (the default): automatic per frame, 320
                                while the frame's mean list length is at most 450 entries, no
                                split above; the image does not depend on it beyond fp32
                                reassociation of T                                              */
} h3dgs_render_opts;

/* Counters of the most recent h3dgs_render (read with a stream synchronisation). */
typedef struct {
    int64_t n_cut;        /* cut nodes rendered (all cameras)                    */
    int64_t n_visible;    /* splats surviving culling                            */
    int64_t n_pairs;      /* (tile, splat) pairs after binning                   */
    int64_t n_tiles;      /* tiles over all cameras                              */
    int64_t n_pixels;     /* pixels over all cameras                             */
    uint32_t device_flags; /* bit 0: pair capacity exceeded, bit 1: splat capacity
                              exceeded, bit 2: cut truncated to capacity, bit 3: a
                              bounded wait of one thread block on another (sort,
                              scan or blend queue) gave up: the frame is invalid,
                              the context stays usable; bit 7: a bounds check of a
                              checked build (h3dgs_build_flags) failed: the file and
                              line are in h3dgs_last_error                        */
    int64_t n_evals;      /* (pixel, splat) evaluations of the blend's main pass
                             (counted only at profiling level 2, else 0)        */
    int64_t n_evals_tpass; /* extra evaluations: the walks of the middle chunks' producers
                             of split tiles, which the consumers repeat while counting
                             (likewise)                                          */
    int64_t n_items;      /* blend work items (tiles, split tiles count once per chunk) */
    int64_t n_evals_interp; /* main-pass evaluations of splats with an interpolated parent
                               (t != 0, Eq. alphap evaluated too; profiling level 2, else 0) */
    int64_t n_contrib;    /* (pixel, splat) pairs whose colour was accumulated: alpha at or above the
                             floor, before the transmittance stop (profiling level 2, else 0) */
    int64_t n_contrib_interp; /* those of splats with an interpolated parent (t != 0; likewise) */
    int64_t n_cut_visited; /* nodes whose record the last cut read: for the one-camera scan all nodes
                              except those of the 256-node rows it skipped (a row is skipped when a
                              bound on its nodes' parents' granularity is below tau, so none of its
                              nodes can be in the cut), for a camera batch all nodes, for the
                              traversal the cut and its ancestors (h3dgs_set_cut_mode) */
} h3dgs_stats;

/* Per-stage device times of the most recent select_cut / render / render_backward, in ms,
 * measured with CUDA events on the context's stream while profiling is enabled. */
typedef enum {
    H3DGS_STAGE_CUT = 0,        /* a1 + a2: mark, scans, ordered compaction          */
    H3DGS_STAGE_PREPROCESS,     /* a3 + a4: interpolate, project, SH                 */
    H3DGS_STAGE_DEPTH_SORT,     /* a5: depth radix sort of the splats                */
    H3DGS_STAGE_DUPLICATE,      /* a5: pair-offset scan and (tile, splat) emission   */
    H3DGS_STAGE_TILE_SORT,      /* a5: stable radix sort of the pairs by tile        */
    H3DGS_STAGE_RANGES,         /* a6: tile ranges (marked by the tile sort's last pass:
                                   0; the stage is kept for the layout of the times) */
    H3DGS_STAGE_BLEND,          /* a7: per-tile blend                                */
    H3DGS_STAGE_BACKWARD_BLEND, /* a8: reverse per-tile blend                        */
    H3DGS_STAGE_BACKWARD_SPLAT, /* a8: projection/interpolation adjoint and scatter  */
    H3DGS_STAGE_BLEND_QUEUE,    /* a7: the blend's main kernel alone (inside BLEND)  */
    H3DGS_STAGE_COUNT
} h3dgs_stage;

/* ------------------------------------------------------------------------------ lifecycle */

/* Create a context on CUDA device `device`, issuing all work on `cuda_stream` (a cudaStream_t;
 * NULL = the legacy default stream).  Fails with H3DGS_ERR_NO_DEVICE when no device exists or it
 * is not compute capability 10.3.  *out receives the context (NULL on failure). */
h3dgs_status h3dgs_create(h3dgs_ctx** out, int32_t device, void* cuda_stream);

/* Destroy a context and free its workspace (synchronises its stream).  NULL is accepted. */
h3dgs_status h3dgs_destroy(h3dgs_ctx* ctx);

/* Message of the last failed call on this context (never NULL; "" after success). */
const char* h3dgs_last_error(const h3dgs_ctx* ctx);

/* Fill *opts with the defaults listed in h3dgs_render_opts. */
void h3dgs_default_opts(h3dgs_render_opts* opts);

/* Fix the workspace capacities (cut-node splats and tile pairs over all cameras of one render)
 * and switch the context to fixed-capacity mode: h3dgs_render then never synchronises, so it can
 * be captured in a CUDA graph.  Overflow sets h3dgs_stats.device_flags bit 0 and the frame is
 * incomplete.  Passing 0 for both returns to the default mode, in which h3dgs_render reads the
 * pair count back once per call and grows its workspace as needed.  Synchronous. */
h3dgs_status h3dgs_reserve(h3dgs_ctx* ctx, int64_t max_splats, int64_t max_pairs);

/* ------------------------------------------------------------------------------ hierarchy */

/* Writable node arrays (device), the layouts of h3dgs_hierarchy, sized for 2L - 1 nodes. */
typedef struct {
    float *mean, *scale, *rot, *opacity, *sh, *box_min, *box_max;
    int32_t *parent, *child_start, *child_count;
} h3dgs_node_arrays;

/* Build the hierarchy over n_leaves leaf Gaussians on the device (Sec. 4.1): leaf boxes are the
 * AABBs of the 3-sigma ellipsoids; groups are split top-down at the median of the members'
 * means projected on the longest axis of the group's box (ties to the lower axis; members
 * ordered by (projected mean, leaf index); the left child takes floor(n/2)); interior nodes
 * are merged bottom-up from their two children with Eq. merge, weights w'_i = o_i S_i (S_i the
 * ellipsoid surface, Thomsen's formula), SH merged with the same weights and the parent
 * opacity set to the falloff sum(w'_i) / S_p; then, from the root down, each child's axes are
 * reinterpreted by the proper signed axis permutation minimising its rotation relative to its
 * parent (orientation matching, Sec. 4.2).  Nodes are numbered breadth-first.  Attributes are
 * computed in fp64 and rounded to fp32 once.  Inputs are device arrays in the layouts of
 * h3dgs_hierarchy ([L,3], [L,3], [L,4], [L], [L,48]); `out` receives 2 n_leaves - 1 nodes.
 * Synchronous; allocates temporary device memory (about 500 bytes per node).
 * Errors: INVALID_ARG (n_leaves < 1 or > 2^30, NULL or misaligned pointers), OOM, CUDA. */
h3dgs_status h3dgs_build_hierarchy(h3dgs_ctx* ctx, int64_t n_leaves, const float* mean, const float* scale,
                                   const float* rot, const float* opacity, const float* sh,
                                   const h3dgs_node_arrays* out);

/* Consolidated hierarchy over a chunked scene (the chunk-wise build and consolidation of large
 * captures, Sec. 6): the leaves are grouped into n_chunks chunks (chunk c = leaves
 * [chunk_offsets[c], chunk_offsets[c + 1]), host array of n_chunks + 1 ascending offsets starting at
 * 0); every chunk gets its own hierarchy exactly as h3dgs_build_hierarchy builds it from the chunk's
 * leaves alone, and a top tree built the same way over the chunk roots joins them (its leaf boxes
 * are the chunks' leaf-union boxes, its leaves are the chunk roots; the chunk roots keep their own
 * frames, i.e. orientation matching stops at the chunk boundary).  Node order: the top tree's
 * 2 n_chunks - 1 nodes breadth-first, then chunk after chunk that chunk's nodes except its root in
 * the chunk's own breadth-first order; every parent precedes its children and children are
 * contiguous.  `out` receives 2 L - 1 nodes for L leaves in total.  Synchronous; allocates
 * temporary device memory.  Errors: INVALID_ARG (bad offsets, an empty chunk, NULL or misaligned
 * pointers), OOM, CUDA. */
h3dgs_status h3dgs_build_hierarchy_chunked(h3dgs_ctx* ctx, int32_t n_chunks, const int64_t* chunk_offsets,
                                           const float* mean, const float* scale, const float* rot,
                                           const float* opacity, const float* sh, const h3dgs_node_arrays* out);

/* Compaction of the resident hierarchy (Sec. 5.2) for a set of training views.  The leaves start
 * out marked; for tau = tau_min, 2 tau_min, 4 tau_min, ... (doubled in fp32) while tau <= tau_max,
 * the bottom-most nodes of the union of the views' cuts at tau (the cut rule of h3dgs_select_cut,
 * with each camera's own tau ignored) are marked and every unmarked node strictly below them is
 * removed.  A kept node's parent becomes its closest kept ancestor, so nodes may end up with
 * K > 2 children (the transition opacity then uses 1 - (1 - alpha_p)^(1/K)).  The kept nodes are
 * renumbered breadth-first from the root, siblings in their old relative order; attributes and
 * boxes are copied unchanged.  cams: HOST array of 1 .. 2^20 cameras (only R, T, fx, fy are used).
 * out: device arrays with room for `capacity` nodes, 16-byte aligned, not overlapping the resident
 * hierarchy; old_index (device, nullable, [capacity]) receives the old index of every new node;
 * *n_out (host) the number of kept nodes.  The resident hierarchy is not changed (upload the
 * result to use it).  Requires nested boxes (a parent's box contains its children's), as built by
 * h3dgs_build_hierarchy.  Synchronous; allocates temporary device memory (about 40 bytes per node).
 * Errors: STATE (no hierarchy), INVALID_ARG (tau_min <= 0, a non-finite tau, more than 64 levels,
 * bad cameras, NULL, misaligned or overlapping arrays, a parent index not below its child's),
 * CAPACITY (*n_out > capacity; nothing written), TIMEOUT, OOM, CUDA. */
h3dgs_status h3dgs_compact_hierarchy(h3dgs_ctx* ctx, const h3dgs_camera* cams, int32_t n_cams, float tau_min,
                                     float tau_max, const h3dgs_node_arrays* out, int64_t capacity,
                                     int32_t* old_index, int64_t* n_out);

/* a0 -- make a hierarchy resident.  The arrays are BORROWED: they must stay allocated, and the
 * topology and boxes unchanged, until the next upload or h3dgs_destroy.  Attributes (mean, scale,
 * rot, opacity, sh) may be updated in place between calls (e.g. by an optimiser).  The library
 * derives a packed 32-byte record per node (box + parent + child count) for the cut kernels.
 * Errors: INVALID_ARG on NULL pointers, n_nodes < 1 or > 2^31 - 1, misaligned pointers.
 * The topology is trusted (not validated on the device). */
h3dgs_status h3dgs_upload_hierarchy(h3dgs_ctx* ctx, const h3dgs_hierarchy* hier);

/* Streamed (out-of-core) hierarchy (Sec. 6.3: the cut is updated every few frames by transferring
 * the nodes it needs from CPU RAM to the GPU; a cleanup runs every 100 frames).  Like
 * h3dgs_upload_hierarchy, but the attribute arrays (mean, scale, rot, opacity, sh) are PAGE-LOCKED
 * HOST arrays (cudaHostAlloc / cudaHostRegister; borrowed, same layouts) while the boxes and the
 * topology are device arrays.  The library keeps the 32-byte cut records of every node on the
 * device and a cache of `cache_nodes` attribute rows (236 bytes each).  h3dgs_select_cut works as
 * usual; before a cut is rendered, h3dgs_stream_update must have made its nodes resident.  Renders
 * read attributes from the cache and are bit-identical to a resident hierarchy's; a cut node that
 * is not resident is left out of the frame and sets bit 5 (0x20) of h3dgs_stats.device_flags.
 * h3dgs_render_backward and h3dgs_compact_hierarchy return STATE on a streamed hierarchy; any
 * upload replaces it.  Errors: INVALID_ARG (host attributes not page-locked, boxes/topology not
 * device memory, sizes), OOM, CUDA. */
h3dgs_status h3dgs_upload_hierarchy_streamed(h3dgs_ctx* ctx, const h3dgs_hierarchy* hier, int64_t cache_nodes);

/* Makes every node of a cut (as returned by h3dgs_select_cut for n_cams cameras) and the parent of
 * every entry with t != 0 resident, stamped with `frame`: absent nodes get free cache rows and are
 * copied from host memory by a device gather over the host link.  *n_transferred (host, nullable;
 * when given the call synchronises) = the number of nodes copied.  When the free rows run out the
 * remaining nodes stay absent, bit 6 (0x40) of device_flags is set and, if n_transferred is given,
 * the call returns CAPACITY.  Asynchronous and graph-capturable when n_transferred is NULL. */
h3dgs_status h3dgs_stream_update(h3dgs_ctx* ctx, int32_t n_cams, const int32_t* cut_ids, const float* cut_t,
                                 const int64_t* cut_offsets, int32_t frame, int64_t* n_transferred);

/* Cleanup: frees the cache row of every resident node whose last update stamp s has
 * frame - s > max_age.  *n_resident (host, nullable; synchronises) = the rows still in use. */
h3dgs_status h3dgs_stream_cleanup(h3dgs_ctx* ctx, int32_t frame, int32_t max_age, int64_t* n_resident);

/* ------------------------------------------------------------------------------ per frame */

/* a1 + a2 -- cut selection and interpolation weights (Sec. 4.2, Fig. gran-cut, Eq. t_interp).
 * For each camera k (cams: HOST array of n_cams, 1 <= n_cams <= 4096):
 *   granularity eps(n) = f * size(n) / dist(n), where f = max(fx, fy), size(n) is the largest
 *   side of the node's box and dist(n) the distance from the camera centre c = -R^T T to the
 *   closest point of the box (+inf when c is inside the box);
 *   n is in the cut  <=>  (eps(n) < tau or n is a leaf) and (n is the root or eps(parent) >= tau);
 *   the parent weight t = (tau - eps(n)) / (eps(parent) - eps(n)) for nodes that passed the test
 *   with a finite eps(parent), else 0 (root, leaves forced in, camera inside the parent box).
 * Outputs (device): cut_ids[cut_offsets[k] .. cut_offsets[k+1]) = the cut of camera k in
 * ascending node order; cut_t (nullable) the matching t; cut_offsets [n_cams + 1] (int64).
 * At most `capacity` ids are written over all cameras; offsets are clamped to capacity.  If
 * total_out (host) is non-NULL the call synchronises, stores the untruncated total there and
 * returns H3DGS_ERR_CAPACITY when it exceeded capacity; with total_out NULL it does not
 * synchronise and truncation is silent. */
h3dgs_status h3dgs_select_cut(h3dgs_ctx* ctx, const h3dgs_camera* cams, int32_t n_cams,
                              int32_t* cut_ids, float* cut_t, int64_t* cut_offsets, int64_t capacity,
                              int64_t* total_out);

/* How h3dgs_select_cut finds one camera's cut (camera batches always scan):
 *   0 (default): the scan, currently the faster choice at every size measured (up to 100M nodes);
 *   1 the scan: every node's record is tested (one pass, decoupled look-back);
 *   2 the traversal: a level-by-level descent from the root reads only the records of the cut and its
 *     ancestors (a cooperative launch with a bounded grid barrier per level), then an ordered
 *     compaction of per-node marks writes the ids ascending.  Same cut and weights as the scan for
 *     trees whose boxes nest (granularity never larger at a child than at its parent, Sec. 4.2).
 * Works for trees up to 1024 levels deep (deeper: device flag bit 2, the cut is incomplete).  The
 * traversal keeps 4 x 4 B per node of frontier and 4 B per node of weights in the context.
 * Errors: INVALID_ARG for another mode. */
h3dgs_status h3dgs_set_cut_mode(h3dgs_ctx* ctx, int32_t mode);

/* Cut selection that allocates nothing (the paper has no counterpart; this is a deployment aid).
 * For callers that cannot call cudaMalloc: code running under another framework's memory budget or
 * allocator, real-time loops that must not enter the driver's allocator (it may synchronise the
 * device), or processes whose device memory is partitioned up front.  Same rule and outputs as
 * h3dgs_select_cut for ONE camera (cam: host pointer), but it needs no context: it reads the
 * caller's box_min, box_max, parent and child_count arrays directly (other hierarchy fields are
 * ignored) and keeps its scratch in a fixed device array of about 2 MB inside the library.
 *   - hier->n_nodes must be at most H3DGS_NOALLOC_MAX_NODES; larger trees return
 *     H3DGS_ERR_CAPACITY without launching anything.
 *   - The first call on each device looks up the scratch array's device address; make that first
 *     call before any CUDA stream capture on that device.  The address belongs to the device's
 *     current context: when that context changes (after cudaDeviceReset, or when the primary
 *     context was released and created again) the next call looks it up again, so make that call
 *     outside stream capture too.
 *   - All calls in the process share the scratch array: calls whose work overlaps on the GPU
 *     (other streams or host threads) race and must be serialised by the caller.
 *   - Work is issued on `cuda_stream` (cudaStream_t, NULL = legacy default stream) of the current
 *     device.  cut_offsets is device int64[2]; with total_out non-NULL the call synchronises the
 *     stream, stores the untruncated cut size and returns H3DGS_ERR_CAPACITY if it exceeds capacity.
 * No cudaMalloc, cudaFree or other allocating call is made. */
#define H3DGS_NOALLOC_MAX_NODES (1LL << 24)
h3dgs_status h3dgs_select_cut_noalloc(const h3dgs_hierarchy* hier, const h3dgs_camera* cam, int32_t* cut_ids,
                                      float* cut_t, int64_t* cut_offsets, int64_t capacity, int64_t* total_out,
                                      void* cuda_stream);

/* a3 -- export the interpolated attributes of every cut node (Sec. 4.2):
 *   a = (1 - t) a_n + t a_p  (fp32: fmaf(t, a_p, (1 - t) * a_n))  for mean, scale, rot (then
 *   normalised), sh;  the opacities o_n, o_p and the parent's child count K are kept separately.
 * out: device float SoA [62][m_total], rows: mean 0-2, scale 3-5, rot 6-9, sh 10-57, o_n 58,
 * o_p 59, t 60, K 61.  interpolate = 0 forces t = 0.  m_total must equal cut_offsets[n_cams]
 * (host value; the caller knows it from h3dgs_select_cut's total_out). */
h3dgs_status h3dgs_interpolate(h3dgs_ctx* ctx, const h3dgs_camera* cams, int32_t n_cams,
                               const int32_t* cut_ids, const float* cut_t, const int64_t* cut_offsets,
                               int32_t interpolate, float* out, int64_t m_total);

/* a3 .. a7 -- render the cuts of n_cams cameras (HOST array) into `images`: device float,
 * camera k's image [3, H_k, W_k] (planar RGB) starting at offset 3 * sum_{j<k} H_j W_j.
 * Stages (all on the device, no host round trip in fixed-capacity mode):
 *   interpolate + project + SH (EWA: Sigma' = J W Sigma W^T J^T + lowpass I, conic, opacity
 *   compensation, radius ceil(3 sqrt(lambda_max)), tile rectangle), depth sort, duplication into
 *   (tile, splat) pairs, stable tile sort, tile ranges, per-tile front-to-back blend with
 *   alpha = (1 - t) min(c, o_n G) + t alpha'(min(c, o_p G)), alpha' = 1 - (1 - alpha_p)^(1/K)
 *   (Eq. alphap), skipping alpha < alpha_floor and stopping before T would drop below t_min.
 * Each tile's list is ordered by (fp32 view depth, cut position).  cut_t may be NULL (t = 0).
 * save_for_backward = 1 keeps the splats, lists and per-pixel final transmittance for
 * h3dgs_render_backward (valid until the next render or upload).  The backward re-reads cut_ids,
 * cut_t and cut_offsets (borrowed): keep them allocated and unchanged until it has run.
 * Errors: INVALID_ARG (bad cameras/opts), STATE (no hierarchy), OOM, CAPACITY (fixed-capacity
 * mode only reports it through h3dgs_stats.device_flags). */
h3dgs_status h3dgs_render(h3dgs_ctx* ctx, const h3dgs_camera* cams, int32_t n_cams,
                          const int32_t* cut_ids, const float* cut_t, const int64_t* cut_offsets,
                          const h3dgs_render_opts* opts, float* images, int32_t save_for_backward);

/* a8 -- adjoint of the most recent h3dgs_render(save_for_backward = 1) (Sec. 5.1, Sec. 7.1, Sec. 7.3).
 * dL_dimages: device, same packing as `images`.  Gradients are ACCUMULATED into `grads`:
 * node n receives (1 - t) of the gradient of its interpolated mean/scale/rot/sh and its parent p
 * receives t of it (t is a constant); o_n and o_p receive the gradients of their own alpha terms,
 * including d alpha'/d alpha_p = (1/K)(1 - alpha_p)^(1/K - 1); an opacity gradient is zero where
 * its alpha is clamped (Sec. 7.3).  freeze_leaves = 1 leaves the rows of leaf nodes untouched
 * (stop-gradient on leaves, Sec. 7.1).  grads->rot and grads->sh must be 16-byte aligned (they are
 * updated with 4-float vector reductions).  Errors: STATE if no saved forward state, INVALID_ARG for
 * NULL or misaligned gradient arrays. */
h3dgs_status h3dgs_render_backward(h3dgs_ctx* ctx, const float* dL_dimages, const h3dgs_grads* grads,
                                   int32_t freeze_leaves);

/* h3dgs_render with the optional outputs of the appendix's depth regularisation and exposure
 * compensation (h3dgs_render is this call with depth = exposure = NULL):
 *   depth     device float, camera k's [H_k, W_k] at offset sum_{j<k} H_j W_j, or NULL: the expected
 *             depth sum_i T_i alpha_i z_i over the pixel's contributors, z_i the view depth of the
 *             (interpolated) mean, with the same blend decisions as the colour and no background;
 *   exposure  device float [n_cams][12], or NULL: camera k's row-major 3x4 affine E_k, applied to
 *             the pixel colour: image = E_k [C + T bg | 1] (the library keeps a copy for the adjoint).
 * Both must be 4-byte aligned.  Errors as h3dgs_render. */
h3dgs_status h3dgs_render_ex(h3dgs_ctx* ctx, const h3dgs_camera* cams, int32_t n_cams,
                             const int32_t* cut_ids, const float* cut_t, const int64_t* cut_offsets,
                             const h3dgs_render_opts* opts, float* images, float* depth, const float* exposure,
                             int32_t save_for_backward);

/* h3dgs_render_backward for a forward made with h3dgs_render_ex: dL_dimages is the gradient of the
 * exposed image (taken back through E_k; E_k itself gets no gradient, it is held fixed as in the
 * paper's hierarchy optimisation) and dL_ddepth (device, the packing of `depth`, or NULL) the
 * gradient of the expected depth, which reaches each splat's alpha and the view depth of its mean.
 * Errors as h3dgs_render_backward, plus STATE when dL_ddepth is given and the forward rendered no
 * depth. */
h3dgs_status h3dgs_render_backward_ex(h3dgs_ctx* ctx, const float* dL_dimages, const float* dL_ddepth,
                                      const h3dgs_grads* grads, int32_t freeze_leaves);

/* ------------------------------------------------------------------------------ inspection */

/* Counters of the last render (synchronises the stream). */
h3dgs_status h3dgs_get_stats(h3dgs_ctx* ctx, h3dgs_stats* out);

/* Profiling level: 0 off; 1 per-stage event timing (every stage bracketed by CUDA events on the
 * context's stream; do not capture such calls in a CUDA graph); 2 timing plus the blend's
 * evaluation counters of h3dgs_stats (which slow the blend down: time with level 1). */
h3dgs_status h3dgs_set_profiling(h3dgs_ctx* ctx, int32_t enable);

/* Calibration of the roofline denominators of the arithmetic-bound kernels on this GPU: chain
 * kernels filling every SM measure the fp32 fused multiply-add rate of the paired instruction the
 * blend uses (*fp32_tflops, 2 flops per FMA) and the exp2 approximation rate (*ex2_gops, results per
 * second / 1e9).  Synchronous, about 20 ms.  Errors: INVALID_ARG (NULL outputs), CUDA. */
h3dgs_status h3dgs_measure_peaks(h3dgs_ctx* ctx, float* fp32_tflops, float* ex2_gops);

/* Stage times (ms) of the last profiled calls, indexed by h3dgs_stage; ms must hold
 * H3DGS_STAGE_COUNT floats (host).  Synchronises the stream.  Stages not run report 0. */
h3dgs_status h3dgs_get_stage_times(h3dgs_ctx* ctx, float* ms);

/* Copy the last render's per-tile lists of camera `cam` to HOST memory (synchronous):
 * ranges [tiles_x * tiles_y][2] = [start, end) into ids; ids = the NODE id of each list entry.
 * *n_out (host) receives the number of entries; at most `cap` ids are written (CAPACITY if
 * more exist). */
h3dgs_status h3dgs_debug_tile_lists(h3dgs_ctx* ctx, int32_t cam, int32_t* ranges, int32_t* ids, int64_t cap,
                                    int64_t* n_out);

/* Copy the last render's splat records to HOST memory (synchronous), one row per cut entry in
 * cut order (all cameras): rec [m][10] = u, v, ca, cb, cc, o_n', o_p', t, K, depth with
 * (ca, cb, cc) the conic scaled so that the base-2 exponent is ca dx^2 + cb dx dy + cc dy^2;
 * rect [m][4] = tile x0, x1, y0, y1 (inclusive), all -1 for culled entries; rgb [m][3]. */
h3dgs_status h3dgs_debug_splats(h3dgs_ctx* ctx, float* rec, int32_t* rect, float* rgb, int64_t m);

/* Test hook for the failure path of the library's bounded waits between thread blocks (the
 * radix-sort and scan look-backs, the blend queue): runs one wait, with the same loop, on a device
 * word that nothing sets, giving up after `polls` polls (1 .. 2^20; each poll sleeps about 0.1 us
 * after the first 32).  Giving up sets bit 3 of h3dgs_stats.device_flags, as a real timeout would;
 * the context stays usable (the next render clears the flag).  Asynchronous on the context's stream.
 * Errors: INVALID_ARG for polls out of range. */
h3dgs_status h3dgs_debug_wait_timeout(h3dgs_ctx* ctx, int32_t polls);

/* Copy the last render's per-pixel final transmittance and contributor count (the list position
 * after the last contributing splat) to HOST memory for all cameras (synchronous); either output
 * may be NULL.  Only a render with save_for_backward = 1 writes this state (after a forward-only
 * render the arrays hold whatever the last saving render left).  n_pixels must equal the total
 * pixel count of the last render's cameras (INVALID_ARG otherwise); STATE if nothing was rendered. */
h3dgs_status h3dgs_debug_pixel_state(h3dgs_ctx* ctx, float* T_final, int32_t* n_contrib, int64_t n_pixels);

/* Build variant of the loaded library: H3DGS_BUILD_CHECKED when it was compiled with -DH3DGS_CHECK
 * (libh3dgs_check.so): every index taken from data (parent and cut ids, list entries, radix staging
 * slots and scatter destinations, work items) is range-checked before its access in the cut,
 * preprocess, sort, blend and adjoint kernels; a failure skips the access, never traps, and sets
 * bit 7 of h3dgs_stats.device_flags (the file and line in h3dgs_last_error).  A debug aid standing
 * in for a memory checker; 0 for the default build, whose checks compile away. */
#define H3DGS_BUILD_CHECKED 1
int32_t h3dgs_build_flags(void);

#ifdef __cplusplus
}
#endif

#endif /* H3DGS_H */
