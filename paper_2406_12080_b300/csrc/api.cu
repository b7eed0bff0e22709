// C ABI of libh3dgs: context, workspace and the orchestration of the per-frame stages.
// Every stage runs in this library's kernels; host code only validates arguments, does integer
// bookkeeping (tile grids, offsets) and manages device memory.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "internal.cuh"

using namespace h3dgs;

namespace {

struct DBuf {
    void* p = nullptr;
    size_t n = 0;
};

cudaError_t ensure(DBuf& b, size_t bytes) {
    if (bytes <= b.n && b.p) return cudaSuccess;
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.n = 0;
    size_t nb = std::max<size_t>(bytes + bytes / 4, 256);
    cudaError_t e = cudaMalloc(&b.p, nb);
    if (e != cudaSuccess) {
        b.p = nullptr;
        return e;
    }
    b.n = nb;
    return cudaSuccess;
}

template <typename T>
T* P(DBuf& b) { return reinterpret_cast<T*>(b.p); }

// device counter block
// C_EVALS, C_EVALS_T, C_EVALS_I, C_CONTRIB and C_CONTRIB_I occupy two words each (64-bit counters, in this order)
// C_NSORTED: a zero word (the bounded-wait probe); C_NTSORT: unused
// C_NITEMS: 4 words (items, producers, singles, split tiles).  C_FLAGS: render flags (cleared by every render);
// C_CUTFLAGS: cut flags (cleared by every cut); the stats report both.  C_CUTSKIP: nodes in the rows
// the one-camera scan skipped (cleared by every cut).
enum { C_FLAGS = 0, C_NSPLATS = 1, C_NVISIBLE = 2, C_NPAIRS = 3, C_NPAIRS_KEPT = 4, C_NSORTED = 6,
       C_NTSORT = 7, C_NITEMS = 14, C_CUTFLAGS = 18, C_CUTSKIP = 19, C_EVALS = 20, C_EVALS_T = 22, C_EVALS_I = 24, C_CONTRIB = 26,
       C_CONTRIB_I = 28, C_COUNT = 30 };
constexpr int EVAL_WORDS = 10;   // the five 64-bit blend counters from C_EVALS on

}  // namespace

struct h3dgs_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    std::string err;
    int num_sms = 148;
    h3dgs_hierarchy hier{};
    bool has_hier = false;
    DBuf rec, rec_tb, cams, counters;
    DBuf cut_mask, cut_bc, cut_tot, cut_lb;
    // traversal cut: frontiers, their parents' granularities, level counts + barrier, marks, weights
    DBuf tr_front0, tr_front1, tr_feps0, tr_feps1, tr_level, tr_mark, tr_tnode;
    int cut_mode = 0;            // 0 (default) and 1: the scan; 2: the traversal
    int tr_grid = -1;            // resident blocks of the cooperative descent (-1: not yet queried)
    size_t tr_mark_bytes = 0;    // zeroed size of tr_mark
    bool last_cut_traversed = false;
    DBuf s_rec, s_rect, s_key, s_idx, s_key2, s_idx2, s_key3, s_tiles, s_poff;
    DBuf pk0, pv0, pk1, pv1, ranges;
    DBuf sortw, seg_start, hists;   // hists: [2][4][256] digit histograms of the depth and tile keys
    DBuf fw;                        // fixed-capacity frame workspace (all cleared by one launch per render)
    DBuf T_final, n_contrib, splat_grad;
    DBuf items, q_prod, q_single, q_cons, queue_sync, tile_item0, tile_nch, sc_Tc, sc_C, sc_Tend, sc_last, sc_D;
    DBuf exposure;   // copy of the last render's exposure affines [n_cams][12]
    // streamed hierarchy (attributes in host memory, a device cache of rows)
    bool streamed = false;
    StreamState st{};
    DBuf st_mean, st_scale, st_rot, st_opacity, st_sh, st_slot_of, st_node_of, st_stamp, st_free, st_missing, st_count;
    int64_t item_cap = 0;
    bool fixed = false;
    int64_t cap_splats = 0, cap_pairs = 0;
    // state of the last render
    bool rendered = false, saved = false, saved_depth = false, has_exposure = false;
    std::vector<h3dgs_camera> cams_host;
    std::vector<int64_t> tile_base, pix_base;
    std::vector<int32_t> tiles_x, tiles_y;
    int64_t n_tiles = 0, n_pixels = 0, splat_cap_used = 0, pair_cap_used = 0;
    DevOpts opts{};
    const int32_t* cut_ids = nullptr;
    const float* cut_t = nullptr;
    const int64_t* cut_offsets = nullptr;
    bool pairs_in_1 = false;
    // profiling
    bool prof = false;
    bool count = false;   // blend evaluation counters (profiling level 2)
    cudaEvent_t ev[2 * H3DGS_STAGE_COUNT] = {};
    bool ev_used[H3DGS_STAGE_COUNT] = {};
};

namespace {

h3dgs_status fail(h3dgs_ctx* c, h3dgs_status s, const std::string& msg) {
    if (c) c->err = msg;
    return s;
}

h3dgs_status cuda_fail(h3dgs_ctx* c, cudaError_t e, const char* where) {
    return fail(c, e == cudaErrorMemoryAllocation ? H3DGS_ERR_OOM : H3DGS_ERR_CUDA,
                std::string(where) + ": " + cudaGetErrorString(e));
}

// stage brackets (only while profiling)
void stage_begin(h3dgs_ctx* ctx, int st) {
    if (ctx->prof) cudaEventRecord(ctx->ev[2 * st], ctx->stream);
}
void stage_end(h3dgs_ctx* ctx, int st) {
    if (ctx->prof) {
        cudaEventRecord(ctx->ev[2 * st + 1], ctx->stream);
        ctx->ev_used[st] = true;
    }
}

#define CK(expr, where)                                        \
    do {                                                       \
        cudaError_t e_ = (expr);                               \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, where); \
    } while (0)

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

h3dgs_status check_cams(h3dgs_ctx* ctx, const h3dgs_camera* cams, int32_t n_cams) {
    if (!cams || n_cams < 1 || n_cams > MAX_CAMS) return fail(ctx, H3DGS_ERR_INVALID_ARG, "cams: need 1..4096 cameras");
    for (int i = 0; i < n_cams; ++i) {
        const h3dgs_camera& c = cams[i];
        if (c.width < 1 || c.height < 1 || c.width > 16384 || c.height > 16384)
            return fail(ctx, H3DGS_ERR_INVALID_ARG, "camera " + std::to_string(i) + ": image size out of range");
        if (!(c.fx > 0) || !(c.fy > 0) || !(c.znear > 0) || !(c.tau >= 0))
            return fail(ctx, H3DGS_ERR_INVALID_ARG, "camera " + std::to_string(i) + ": fx, fy, znear > 0 and tau >= 0");
    }
    return H3DGS_OK;
}

// Upload cameras with their tile grids; fills the ctx bookkeeping vectors.
// defer (nullable): a single batch is returned there for a later launch to set up, instead of launched
h3dgs_status setup_cameras(h3dgs_ctx* ctx, const h3dgs_camera* cams, int32_t n_cams, int tile_w, int tile_h,
                           CamBatch* defer = nullptr) {
    CK(ensure(ctx->cams, sizeof(DevCam) * (size_t)n_cams), "camera buffer");
    ctx->cams_host.assign(cams, cams + n_cams);
    ctx->tile_base.resize(n_cams);
    ctx->pix_base.resize(n_cams);
    ctx->tiles_x.resize(n_cams);
    ctx->tiles_y.resize(n_cams);
    int64_t tb = 0, pb = 0;
    for (int i = 0; i < n_cams; ++i) {
        ctx->tiles_x[i] = (cams[i].width + tile_w - 1) / tile_w;
        ctx->tiles_y[i] = (cams[i].height + tile_h - 1) / tile_h;
        ctx->tile_base[i] = tb;
        ctx->pix_base[i] = pb;
        tb += (int64_t)ctx->tiles_x[i] * ctx->tiles_y[i];
        pb += (int64_t)cams[i].width * cams[i].height;
    }
    ctx->n_tiles = tb;
    ctx->n_pixels = pb;
    for (int first = 0; first < n_cams; first += CAM_BATCH) {
        CamBatch b;
        std::memset(&b, 0, sizeof(b));
        b.first = first;
        b.count = std::min(CAM_BATCH, n_cams - first);
        for (int i = 0; i < b.count; ++i) {
            b.cam[i] = cams[first + i];
            b.tiles_x[i] = ctx->tiles_x[first + i];
            b.tiles_y[i] = ctx->tiles_y[first + i];
            b.tile_base[i] = ctx->tile_base[first + i];
            b.pix_base[i] = ctx->pix_base[first + i];
        }
        if (defer && n_cams <= CAM_BATCH) {
            *defer = b;
            break;
        }
        CK(launch_camera_setup(b, nullptr, P<DevCam>(ctx->cams), ctx->stream), "camera set-up");
    }
    return H3DGS_OK;
}

DevHier dev_hier(h3dgs_ctx* ctx) {
    DevHier h;
    h.n = ctx->hier.n_nodes;
    h.mean = ctx->hier.mean;
    h.scale = ctx->hier.scale;
    h.rot = reinterpret_cast<const float4*>(ctx->hier.rot);
    h.opacity = ctx->hier.opacity;
    h.sh = reinterpret_cast<const float4*>(ctx->hier.sh);
    h.parent = ctx->hier.parent;
    h.child_count = ctx->hier.child_count;
    h.rec = P<const float4>(ctx->rec);
    h.row_bound = P<const float4>(ctx->rec_tb);
    h.row_of = nullptr;
    if (ctx->streamed) {
        h.mean = ctx->st.mean;
        h.scale = ctx->st.scale;
        h.rot = reinterpret_cast<const float4*>(ctx->st.rot);
        h.opacity = ctx->st.opacity;
        h.sh = reinterpret_cast<const float4*>(ctx->st.sh);
        h.row_of = ctx->st.slot_of;
    }
    return h;
}

DevOpts dev_opts(const h3dgs_render_opts& o) {
    DevOpts d;
    d.tile_w = o.tile_w; d.tile_h = o.tile_h; d.lowpass = o.lowpass; d.alpha_clamp = o.alpha_clamp;
    d.alpha_floor = o.alpha_floor; d.t_min = o.t_min; d.aa_compensate = o.aa_compensate;
    d.interpolate = o.interpolate;
    d.chunk = o.blend_chunk > 0 ? o.blend_chunk : 0;   // 0: automatic (the plan picks it per frame)
    for (int i = 0; i < 3; ++i) d.bg[i] = o.bg[i];
    return d;
}

bool supported_tile(int w, int h) {
    return (w == 16 && h == 16) || (w == 8 && h == 8) || (w == 32 && h == 8) || (w == 8 && h == 32) ||
           (w == 16 && h == 8);
}


}  // namespace

// (outside the anonymous namespace: needs the full context type)
static BlendArgs blend_args(h3dgs_ctx* ctx, int n_cams, float* images, float* depth) {
    BlendArgs a;
    a.cams = P<DevCam>(ctx->cams);
    a.n_cams = n_cams;
    a.n_tiles = ctx->n_tiles;
    a.o = ctx->opts;
    a.ranges = P<int2>(ctx->ranges);
    a.list = ctx->pairs_in_1 ? P<uint32_t>(ctx->pv1) : P<uint32_t>(ctx->pv0);
    a.splat = P<float4>(ctx->s_rec);
    a.n_splats = P<uint32_t>(ctx->counters) + C_NSPLATS;
    a.chunk = ctx->opts.chunk;
    a.n_pairs = P<uint32_t>(ctx->counters) + C_NPAIRS_KEPT;
    a.item_cap = ctx->item_cap;
    a.items = P<int2>(ctx->items);
    a.q_prod = P<uint32_t>(ctx->q_prod);
    a.q_single = P<uint32_t>(ctx->q_single);
    a.q_cons = P<uint32_t>(ctx->q_cons);
    a.queue_sync = P<uint32_t>(ctx->queue_sync);
    a.tile_item0 = P<int32_t>(ctx->tile_item0);
    a.tile_nch = P<int32_t>(ctx->tile_nch);
    a.num_sms = ctx->num_sms;
    a.n_items = P<uint32_t>(ctx->counters) + C_NITEMS;
    a.scratch_Tc = P<float>(ctx->sc_Tc);
    a.scratch_C = P<float>(ctx->sc_C);
    a.scratch_Tend = P<float>(ctx->sc_Tend);
    a.scratch_last = P<int32_t>(ctx->sc_last);
    a.images = images;
    a.depth = depth;
    a.exposure = ctx->has_exposure ? P<const float>(ctx->exposure) : nullptr;
    a.scratch_D = P<float>(ctx->sc_D);
    a.T_final = P<float>(ctx->T_final);
    a.n_contrib = P<int32_t>(ctx->n_contrib);
    // evaluation counters only at profiling level 2 (counting costs instructions in the blend's inner loop)
    a.n_evals = ctx->count ? reinterpret_cast<unsigned long long*>(P<uint32_t>(ctx->counters) + C_EVALS) : nullptr;
    a.work = P<uint32_t>(ctx->sortw);
    a.work_words = ctx->sortw.n / sizeof(uint32_t);
    a.flags = P<uint32_t>(ctx->counters) + C_FLAGS;
    a.ev_queue = nullptr;
    a.pre_zeroed = false;
    return a;
}

namespace {

// Sort and scan workspace for sorts of up to n_cap keys (grown here; no growth once reserved).
cudaError_t sort_work(h3dgs_ctx* ctx, int64_t n_cap, SortWork* w) {
    const size_t words = radix_work_words(n_cap);
    cudaError_t e = ensure(ctx->sortw, sizeof(uint32_t) * words);
    if (e != cudaSuccess) return e;
    w->work = P<uint32_t>(ctx->sortw);
    w->words = ctx->sortw.n / sizeof(uint32_t);
    w->num_sms = ctx->num_sms;
    w->flags = P<uint32_t>(ctx->counters) + C_FLAGS;
    return cudaSuccess;
}

// A build is synchronous: a sort wait that gave up is reported as its status.
h3dgs_status check_build_flags(h3dgs_ctx* ctx) {
    uint32_t f = 0;
    CK(cudaMemcpyAsync(&f, P<uint32_t>(ctx->counters) + C_FLAGS, sizeof(f), cudaMemcpyDeviceToHost, ctx->stream),
       "read flags");
    CK(cudaStreamSynchronize(ctx->stream), "build sync");
    if (f & FLAG_WAIT_TIMEOUT) return fail(ctx, H3DGS_ERR_TIMEOUT, "build: a bounded wait between blocks gave up");
    return H3DGS_OK;
}

}  // namespace

extern "C" {

h3dgs_status h3dgs_create(h3dgs_ctx** out, int32_t device, void* cuda_stream) {
    if (!out) return H3DGS_ERR_INVALID_ARG;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || n <= device || device < 0) {
        cudaGetLastError();
        return H3DGS_ERR_NO_DEVICE;
    }
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return H3DGS_ERR_NO_DEVICE;
    if (!(prop.major == 10 && prop.minor == 3)) return H3DGS_ERR_NO_DEVICE;
    if (cudaSetDevice(device) != cudaSuccess) return H3DGS_ERR_NO_DEVICE;
    h3dgs_ctx* ctx = new h3dgs_ctx();
    ctx->device = device;
    ctx->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
    ctx->num_sms = prop.multiProcessorCount;
    cudaError_t e = ensure(ctx->counters, sizeof(uint32_t) * C_COUNT);
    if (e == cudaSuccess) e = cudaMemset(ctx->counters.p, 0, sizeof(uint32_t) * C_COUNT);
    if (e != cudaSuccess) {
        h3dgs_destroy(ctx);
        return e == cudaErrorMemoryAllocation ? H3DGS_ERR_OOM : H3DGS_ERR_CUDA;
    }
    *out = ctx;
    return H3DGS_OK;
}

h3dgs_status h3dgs_destroy(h3dgs_ctx* ctx) {
    if (!ctx) return H3DGS_OK;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    DBuf* bufs[] = {&ctx->rec, &ctx->rec_tb, &ctx->cams, &ctx->counters, &ctx->cut_mask, &ctx->cut_bc, &ctx->cut_tot, &ctx->cut_lb,
                    &ctx->s_rec, &ctx->s_rect, &ctx->s_key, &ctx->s_idx, &ctx->s_key2, &ctx->s_idx2,
                    &ctx->s_key3, &ctx->s_tiles, &ctx->s_poff, &ctx->pk0, &ctx->pv0, &ctx->pk1, &ctx->pv1,
                    &ctx->ranges, &ctx->sortw, &ctx->seg_start, &ctx->hists, &ctx->fw, &ctx->T_final, &ctx->n_contrib, &ctx->splat_grad,
                    &ctx->items, &ctx->q_prod, &ctx->q_single, &ctx->q_cons, &ctx->queue_sync,
                    &ctx->tile_item0, &ctx->tile_nch, &ctx->sc_Tc, &ctx->sc_C, &ctx->sc_Tend,
                    &ctx->sc_last, &ctx->sc_D, &ctx->exposure, &ctx->st_mean, &ctx->st_scale, &ctx->st_rot,
                    &ctx->st_opacity, &ctx->st_sh, &ctx->st_slot_of, &ctx->st_node_of, &ctx->st_stamp,
                    &ctx->st_free, &ctx->st_missing, &ctx->st_count, &ctx->tr_front0, &ctx->tr_front1,
                    &ctx->tr_feps0, &ctx->tr_feps1, &ctx->tr_level, &ctx->tr_mark, &ctx->tr_tnode};
    for (DBuf* b : bufs)
        if (b->p) cudaFree(b->p);
    for (auto& e : ctx->ev)
        if (e) cudaEventDestroy(e);
    delete ctx;
    return H3DGS_OK;
}

const char* h3dgs_last_error(const h3dgs_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

void h3dgs_default_opts(h3dgs_render_opts* o) {
    if (!o) return;
    o->tile_w = 16;
    o->tile_h = 16;
    o->lowpass = 0.3f;
    o->alpha_clamp = 0.99f;
    o->alpha_floor = 1.0f / 255.0f;
    o->t_min = 1e-4f;
    o->aa_compensate = 1;
    o->interpolate = 1;
    o->bg[0] = o->bg[1] = o->bg[2] = 0.0f;
    o->blend_chunk = 0;
}

h3dgs_status h3dgs_reserve(h3dgs_ctx* ctx, int64_t max_splats, int64_t max_pairs) {
    if (!ctx) return H3DGS_ERR_INVALID_ARG;
    ctx->err.clear();
    if (max_splats < 0 || max_pairs < 0 || max_pairs > 0xffffffffLL || max_splats > 0x7fffffffLL)
        return fail(ctx, H3DGS_ERR_INVALID_ARG, "reserve: capacities out of range");
    CK(cudaSetDevice(ctx->device), "set device");
    if (max_splats == 0 && max_pairs == 0) {
        ctx->fixed = false;
        return H3DGS_OK;
    }
    const size_t M = (size_t)max_splats, Pn = (size_t)max_pairs;
    CK(ensure(ctx->s_rec, 16 * SPLAT_F4 * M), "splat buffer");
    CK(ensure(ctx->s_rect, 8 * M), "splat buffer");
    DBuf* m4[] = {&ctx->s_key, &ctx->s_idx, &ctx->s_key2, &ctx->s_idx2, &ctx->s_key3, &ctx->s_tiles, &ctx->s_poff};
    for (DBuf* b : m4) CK(ensure(*b, 4 * M), "splat buffer");
    DBuf* p4[] = {&ctx->pk0, &ctx->pv0, &ctx->pk1, &ctx->pv1};
    for (DBuf* b : p4) CK(ensure(*b, 4 * Pn), "pair buffer");
    SortWork w;
    CK(sort_work(ctx, std::max<int64_t>(max_splats, max_pairs), &w), "sort workspace");
    CK(ensure(ctx->seg_start, sizeof(uint32_t) * (size_t)(Pn / DUP_SEG + 2)), "pair segments");
    CK(cudaDeviceSynchronize(), "reserve");
    ctx->fixed = true;
    ctx->cap_splats = max_splats;
    ctx->cap_pairs = max_pairs;
    return H3DGS_OK;
}

h3dgs_status h3dgs_build_hierarchy(h3dgs_ctx* ctx, int64_t L, const float* mean, const float* scale, const float* rot,
                                   const float* opacity, const float* sh, const h3dgs_node_arrays* out) {
    if (!ctx) return H3DGS_ERR_INVALID_ARG;
    ctx->err.clear();
    if (L < 1 || L > (1LL << 30)) return fail(ctx, H3DGS_ERR_INVALID_ARG, "build: n_leaves out of range");
    if (!out) return fail(ctx, H3DGS_ERR_INVALID_ARG, "build: NULL output");
    const void* ptrs[] = {mean, scale, rot, opacity, sh, out->mean, out->scale, out->rot, out->opacity, out->sh,
                          out->box_min, out->box_max, out->parent, out->child_start, out->child_count};
    for (const void* p : ptrs) {
        if (!p) return fail(ctx, H3DGS_ERR_INVALID_ARG, "build: NULL array");
        if (!aligned16(p)) return fail(ctx, H3DGS_ERR_INVALID_ARG, "build: arrays must be 16-byte aligned");
    }
    CK(cudaSetDevice(ctx->device), "set device");
    BuildOut bo{out->mean, out->scale, out->rot, out->opacity, out->sh, out->box_min, out->box_max,
                out->parent, out->child_start, out->child_count};
    SortWork sw;
    CK(sort_work(ctx, L, &sw), "sort workspace");
    CK(cudaMemsetAsync(P<uint32_t>(ctx->counters) + C_FLAGS, 0, sizeof(uint32_t), ctx->stream), "memset");
    CK(build_hierarchy(L, mean, scale, rot, opacity, sh, bo, sw, ctx->num_sms, ctx->stream), "build");
    return check_build_flags(ctx);
}

h3dgs_status h3dgs_build_hierarchy_chunked(h3dgs_ctx* ctx, int32_t n_chunks, const int64_t* off, const float* mean,
                                           const float* scale, const float* rot, const float* opacity, const float* sh,
                                           const h3dgs_node_arrays* out) {
    if (!ctx) return H3DGS_ERR_INVALID_ARG;
    ctx->err.clear();
    if (n_chunks < 1 || !off || off[0] != 0) return fail(ctx, H3DGS_ERR_INVALID_ARG, "build_chunked: bad chunk offsets");
    int64_t Lmax = 0;
    for (int c = 0; c < n_chunks; ++c) {
        if (off[c + 1] <= off[c]) return fail(ctx, H3DGS_ERR_INVALID_ARG, "build_chunked: empty or unordered chunk");
        Lmax = std::max<int64_t>(Lmax, off[c + 1] - off[c]);
    }
    if (off[n_chunks] > (1LL << 30)) return fail(ctx, H3DGS_ERR_INVALID_ARG, "build_chunked: too many leaves");
    if (!out) return fail(ctx, H3DGS_ERR_INVALID_ARG, "build_chunked: NULL output");
    const void* ptrs[] = {mean, scale, rot, opacity, sh, out->mean, out->scale, out->rot, out->opacity, out->sh,
                          out->box_min, out->box_max, out->parent, out->child_start, out->child_count};
    for (const void* p : ptrs) {
        if (!p) return fail(ctx, H3DGS_ERR_INVALID_ARG, "build_chunked: NULL array");
        if (!aligned16(p)) return fail(ctx, H3DGS_ERR_INVALID_ARG, "build_chunked: arrays must be 16-byte aligned");
    }
    CK(cudaSetDevice(ctx->device), "set device");
    BuildOut bo{out->mean, out->scale, out->rot, out->opacity, out->sh, out->box_min, out->box_max,
                out->parent, out->child_start, out->child_count};
    SortWork sw;
    CK(sort_work(ctx, std::max<int64_t>(Lmax, n_chunks), &sw), "sort workspace");
    CK(cudaMemsetAsync(P<uint32_t>(ctx->counters) + C_FLAGS, 0, sizeof(uint32_t), ctx->stream), "memset");
    CK(build_hierarchy_chunked(n_chunks, off, mean, scale, rot, opacity, sh, bo, sw, ctx->num_sms, ctx->stream),
       "build chunked");
    return check_build_flags(ctx);
}

h3dgs_status h3dgs_compact_hierarchy(h3dgs_ctx* ctx, const h3dgs_camera* cams, int32_t n_cams, float tau_min,
                                     float tau_max, const h3dgs_node_arrays* out, int64_t capacity, int32_t* old_index,
                                     int64_t* n_out) {
    if (!ctx) return H3DGS_ERR_INVALID_ARG;
    ctx->err.clear();
    if (!ctx->has_hier) return fail(ctx, H3DGS_ERR_STATE, "compact: no hierarchy uploaded");
    if (ctx->streamed) return fail(ctx, H3DGS_ERR_STATE, "compact: not available for a streamed hierarchy");
    if (!cams || n_cams < 1 || n_cams > (1 << 20)) return fail(ctx, H3DGS_ERR_INVALID_ARG, "compact: need 1..2^20 cameras");
    for (int i = 0; i < n_cams; ++i)
        if (!(cams[i].fx > 0) || !(cams[i].fy > 0) || !std::isfinite(cams[i].fx) || !std::isfinite(cams[i].fy))
            return fail(ctx, H3DGS_ERR_INVALID_ARG, "compact: camera " + std::to_string(i) + " needs finite fx, fy > 0");
    if (!(tau_min > 0) || !std::isfinite(tau_min) || !std::isfinite(tau_max))
        return fail(ctx, H3DGS_ERR_INVALID_ARG, "compact: need tau_min > 0 and a finite tau_max");
    std::vector<float> levels;
    for (float t = tau_min; t <= tau_max; t = t * 2.0f) {
        if (levels.size() == 64) return fail(ctx, H3DGS_ERR_INVALID_ARG, "compact: more than 64 levels");
        levels.push_back(t);
    }
    if (!out || !n_out || capacity < 1) return fail(ctx, H3DGS_ERR_INVALID_ARG, "compact: NULL output or capacity < 1");
    const h3dgs_hierarchy& h = ctx->hier;
    const int64_t N = h.n_nodes;
    const size_t n = (size_t)N;
    struct Range { const void* p; size_t bytes; };
    const Range in[] = {{h.mean, 12 * n}, {h.scale, 12 * n}, {h.rot, 16 * n}, {h.opacity, 4 * n},
                        {h.sh, 192 * n}, {h.box_min, 12 * n}, {h.box_max, 12 * n}, {h.parent, 4 * n},
                        {h.child_start, 4 * n}, {h.child_count, 4 * n}};
    const size_t cap = (size_t)capacity;
    const Range outs[] = {{out->mean, 12 * cap}, {out->scale, 12 * cap}, {out->rot, 16 * cap},
                          {out->opacity, 4 * cap}, {out->sh, 192 * cap}, {out->box_min, 12 * cap},
                          {out->box_max, 12 * cap}, {out->parent, 4 * cap}, {out->child_start, 4 * cap},
                          {out->child_count, 4 * cap}, {old_index, old_index ? 4 * cap : 0}};
    for (const Range& o : outs) {
        if (!o.p && &o != &outs[10]) return fail(ctx, H3DGS_ERR_INVALID_ARG, "compact: NULL output array");
        if (o.p && !aligned16(o.p)) return fail(ctx, H3DGS_ERR_INVALID_ARG, "compact: arrays must be 16-byte aligned");
        const uintptr_t a0 = reinterpret_cast<uintptr_t>(o.p), a1 = a0 + o.bytes;
        for (const Range& i : in) {
            const uintptr_t b0 = reinterpret_cast<uintptr_t>(i.p), b1 = b0 + i.bytes;
            if (o.p && a0 < b1 && b0 < a1)
                return fail(ctx, H3DGS_ERR_INVALID_ARG, "compact: an output overlaps the resident hierarchy");
        }
    }
    CK(cudaSetDevice(ctx->device), "set device");
    SortWork sw;
    CK(sort_work(ctx, N, &sw), "sort workspace");
    CK(cudaMemsetAsync(P<uint32_t>(ctx->counters) + C_FLAGS, 0, sizeof(uint32_t), ctx->stream), "memset");
    BuildOut bo{out->mean, out->scale, out->rot, out->opacity, out->sh, out->box_min, out->box_max,
                out->parent, out->child_start, out->child_count};
    CK(compact_hierarchy(h, P<const float4>(ctx->rec), cams, n_cams, levels.data(), (int)levels.size(), bo, capacity,
                         old_index, n_out, sw, ctx->num_sms, ctx->stream),
       "compact");
    uint32_t f = 0;
    CK(cudaMemcpyAsync(&f, P<uint32_t>(ctx->counters) + C_FLAGS, sizeof(f), cudaMemcpyDeviceToHost, ctx->stream),
       "read flags");
    CK(cudaStreamSynchronize(ctx->stream), "compact sync");
    if (f & FLAG_WAIT_TIMEOUT) return fail(ctx, H3DGS_ERR_TIMEOUT, "compact: a bounded wait between blocks gave up");
    if (f & FLAG_BAD_TOPOLOGY) return fail(ctx, H3DGS_ERR_INVALID_ARG, "compact: a parent index is not below its child's");
    if (*n_out > capacity) return fail(ctx, H3DGS_ERR_CAPACITY, "compact: more kept nodes than capacity");
    return H3DGS_OK;
}

h3dgs_status h3dgs_upload_hierarchy(h3dgs_ctx* ctx, const h3dgs_hierarchy* h) {
    if (!ctx) return H3DGS_ERR_INVALID_ARG;
    ctx->err.clear();
    if (!h) return fail(ctx, H3DGS_ERR_INVALID_ARG, "hierarchy: NULL");
    if (h->n_nodes < 1 || h->n_nodes > 0x7fffffffLL) return fail(ctx, H3DGS_ERR_INVALID_ARG, "hierarchy: n_nodes out of range");
    const void* ptrs[] = {h->mean, h->scale, h->rot, h->opacity, h->sh, h->box_min, h->box_max,
                          h->parent, h->child_start, h->child_count};
    for (const void* p : ptrs) {
        if (!p) return fail(ctx, H3DGS_ERR_INVALID_ARG, "hierarchy: NULL array");
        if (!aligned16(p)) return fail(ctx, H3DGS_ERR_INVALID_ARG, "hierarchy: arrays must be 16-byte aligned");
    }
    CK(cudaSetDevice(ctx->device), "set device");
    CK(ensure(ctx->rec, sizeof(float4) * 2 * (size_t)h->n_nodes), "record buffer");
    CK(launch_pack_records(*h, P<float4>(ctx->rec), ctx->stream), "pack records");
    CK(ensure(ctx->rec_tb, sizeof(float4) * 2 * (size_t)cut_row_count(h->n_nodes)), "row bounds");
    CK(launch_cut_row_bounds(P<const float4>(ctx->rec), h->n_nodes, P<float4>(ctx->rec_tb), ctx->stream), "row bounds");
    ctx->hier = *h;
    ctx->has_hier = true;
    ctx->streamed = false;
    ctx->rendered = ctx->saved = false;
    return H3DGS_OK;
}

h3dgs_status h3dgs_upload_hierarchy_streamed(h3dgs_ctx* ctx, const h3dgs_hierarchy* h, int64_t cache_nodes) {
    if (!ctx) return H3DGS_ERR_INVALID_ARG;
    ctx->err.clear();
    if (!h) return fail(ctx, H3DGS_ERR_INVALID_ARG, "hierarchy: NULL");
    if (h->n_nodes < 1 || h->n_nodes > 0x7fffffffLL) return fail(ctx, H3DGS_ERR_INVALID_ARG, "hierarchy: n_nodes out of range");
    if (cache_nodes < 1 || cache_nodes > 0x7fffffffLL) return fail(ctx, H3DGS_ERR_INVALID_ARG, "stream: cache_nodes out of range");
    CK(cudaSetDevice(ctx->device), "set device");
    const void* dev_ptrs[] = {h->box_min, h->box_max, h->parent, h->child_start, h->child_count};
    for (const void* p : dev_ptrs) {
        cudaPointerAttributes a{};
        if (!p || cudaPointerGetAttributes(&a, p) != cudaSuccess || a.type != cudaMemoryTypeDevice)
            return fail(ctx, H3DGS_ERR_INVALID_ARG, "stream: boxes and topology must be device arrays");
        if (!aligned16(p)) return fail(ctx, H3DGS_ERR_INVALID_ARG, "hierarchy: arrays must be 16-byte aligned");
    }
    const float* host[5] = {h->mean, h->scale, h->rot, h->opacity, h->sh};
    const float* mapped[5];
    for (int k = 0; k < 5; ++k) {
        cudaPointerAttributes a{};
        if (!host[k] || cudaPointerGetAttributes(&a, host[k]) != cudaSuccess || a.type != cudaMemoryTypeHost)
            return fail(ctx, H3DGS_ERR_INVALID_ARG, "stream: attributes must be page-locked host arrays");
        void* d = nullptr;
        if (cudaHostGetDevicePointer(&d, const_cast<float*>(host[k]), 0) != cudaSuccess || !d)
            return fail(ctx, H3DGS_ERR_INVALID_ARG, "stream: attributes not mapped into the device address space");
        mapped[k] = static_cast<const float*>(d);
    }
    const size_t C = (size_t)cache_nodes, N = (size_t)h->n_nodes;
    CK(ensure(ctx->st_mean, 12 * C), "stream cache");
    CK(ensure(ctx->st_scale, 12 * C), "stream cache");
    CK(ensure(ctx->st_rot, 16 * C), "stream cache");
    CK(ensure(ctx->st_opacity, 4 * C), "stream cache");
    CK(ensure(ctx->st_sh, 192 * C), "stream cache");
    CK(ensure(ctx->st_node_of, 4 * C), "stream cache");
    CK(ensure(ctx->st_stamp, 4 * C), "stream cache");
    CK(ensure(ctx->st_free, 4 * C), "stream cache");
    CK(ensure(ctx->st_slot_of, 4 * N), "stream tables");
    CK(ensure(ctx->st_missing, 4 * N), "stream tables");
    CK(ensure(ctx->st_count, 16), "stream tables");
    CK(ensure(ctx->rec, sizeof(float4) * 2 * N), "record buffer");
    CK(launch_pack_records(*h, P<float4>(ctx->rec), ctx->stream), "pack records");
    CK(ensure(ctx->rec_tb, sizeof(float4) * 2 * (size_t)cut_row_count(h->n_nodes)), "row bounds");
    CK(launch_cut_row_bounds(P<const float4>(ctx->rec), h->n_nodes, P<float4>(ctx->rec_tb), ctx->stream), "row bounds");
    StreamState& st = ctx->st;
    st.n_nodes = h->n_nodes;
    st.cap = cache_nodes;
    st.h_mean = mapped[0]; st.h_scale = mapped[1]; st.h_rot = mapped[2]; st.h_opacity = mapped[3]; st.h_sh = mapped[4];
    st.mean = P<float>(ctx->st_mean); st.scale = P<float>(ctx->st_scale); st.rot = P<float>(ctx->st_rot);
    st.opacity = P<float>(ctx->st_opacity); st.sh = P<float>(ctx->st_sh);
    st.slot_of = P<int32_t>(ctx->st_slot_of); st.node_of = P<int32_t>(ctx->st_node_of);
    st.stamp = P<int32_t>(ctx->st_stamp); st.free_list = P<int32_t>(ctx->st_free);
    st.missing = P<int32_t>(ctx->st_missing); st.count = P<uint32_t>(ctx->st_count);
    CK(stream_init(st, ctx->num_sms, ctx->stream), "stream init");
    ctx->hier = *h;
    ctx->has_hier = true;
    ctx->streamed = true;
    ctx->rendered = ctx->saved = false;
    return H3DGS_OK;
}

h3dgs_status h3dgs_stream_update(h3dgs_ctx* ctx, int32_t n_cams, const int32_t* cut_ids, const float* cut_t,
                                 const int64_t* cut_offsets, int32_t frame, int64_t* n_transferred) {
    if (!ctx) return H3DGS_ERR_INVALID_ARG;
    ctx->err.clear();
    if (!ctx->has_hier || !ctx->streamed) return fail(ctx, H3DGS_ERR_STATE, "stream_update: no streamed hierarchy");
    if (n_cams < 1 || n_cams > MAX_CAMS || !cut_ids || !cut_offsets)
        return fail(ctx, H3DGS_ERR_INVALID_ARG, "stream_update: bad cut");
    CK(cudaSetDevice(ctx->device), "set device");
    CK(stream_update(ctx->st, ctx->hier.parent, n_cams, cut_ids, cut_t, cut_offsets, frame,
                     P<uint32_t>(ctx->counters) + C_CUTFLAGS, ctx->num_sms, ctx->stream),
       "stream update");
    if (n_transferred) {
        uint32_t c[4];
        CK(cudaMemcpyAsync(c, ctx->st.count, sizeof(c), cudaMemcpyDeviceToHost, ctx->stream), "read stream counts");
        CK(cudaStreamSynchronize(ctx->stream), "stream sync");
        *n_transferred = c[2];
        if (c[3] > c[2]) return fail(ctx, H3DGS_ERR_CAPACITY, "stream_update: cache full (run a cleanup or enlarge it)");
    }
    return H3DGS_OK;
}

h3dgs_status h3dgs_stream_cleanup(h3dgs_ctx* ctx, int32_t frame, int32_t max_age, int64_t* n_resident) {
    if (!ctx) return H3DGS_ERR_INVALID_ARG;
    ctx->err.clear();
    if (!ctx->has_hier || !ctx->streamed) return fail(ctx, H3DGS_ERR_STATE, "stream_cleanup: no streamed hierarchy");
    if (max_age < 0) return fail(ctx, H3DGS_ERR_INVALID_ARG, "stream_cleanup: max_age < 0");
    CK(cudaSetDevice(ctx->device), "set device");
    CK(stream_cleanup(ctx->st, frame, max_age, ctx->num_sms, ctx->stream), "stream cleanup");
    if (n_resident) {
        uint32_t free_rows = 0;
        CK(cudaMemcpyAsync(&free_rows, ctx->st.count, sizeof(free_rows), cudaMemcpyDeviceToHost, ctx->stream),
           "read stream counts");
        CK(cudaStreamSynchronize(ctx->stream), "stream sync");
        *n_resident = ctx->st.cap - (int64_t)free_rows;
    }
    return H3DGS_OK;
}

h3dgs_status h3dgs_select_cut(h3dgs_ctx* ctx, const h3dgs_camera* cams, int32_t n_cams, int32_t* cut_ids,
                              float* cut_t, int64_t* cut_offsets, int64_t capacity, int64_t* total_out) {
    if (!ctx) return H3DGS_ERR_INVALID_ARG;
    ctx->err.clear();
    if (!ctx->has_hier) return fail(ctx, H3DGS_ERR_STATE, "select_cut: no hierarchy uploaded");
    h3dgs_status st = check_cams(ctx, cams, n_cams);
    if (st != H3DGS_OK) return st;
    if (!cut_offsets || (capacity > 0 && !cut_ids) || capacity < 0)
        return fail(ctx, H3DGS_ERR_INVALID_ARG, "select_cut: NULL output or negative capacity");
    CK(cudaSetDevice(ctx->device), "set device");
    if (n_cams > 1) {   // the one-camera pass derives its camera values itself (no set-up launch)
        st = setup_cameras(ctx, cams, n_cams, 16, 16);
        if (st != H3DGS_OK) return st;
    }
    const int64_t N = ctx->hier.n_nodes;
    CutWork w;
    w.cam0 = cams[0];
    const int64_t max_blocks = (int64_t)ctx->num_sms * 4;
    w.chunk = ((N + max_blocks - 1) / max_blocks + 255) / 256 * 256;
    w.blocks = (int)((N + w.chunk - 1) / w.chunk);
    w.words = (N + 31) / 32;
    CK(ensure(ctx->cut_mask, sizeof(uint32_t) * (size_t)w.words * n_cams), "cut mask");
    CK(ensure(ctx->cut_bc, sizeof(uint32_t) * (size_t)w.blocks * n_cams), "cut counts");
    CK(ensure(ctx->cut_tot, sizeof(int64_t) * (size_t)(n_cams + 1)), "cut totals");
    w.lb_words = (int64_t)cut_single_work_words(N);
    w.num_sms = ctx->num_sms;
    CK(ensure(ctx->cut_lb, sizeof(uint32_t) * (size_t)w.lb_words), "cut look-back");
    w.lb_work = P<uint32_t>(ctx->cut_lb);
    w.mask = P<uint32_t>(ctx->cut_mask);
    w.block_counts = P<uint32_t>(ctx->cut_bc);
    w.cam_totals = P<int64_t>(ctx->cut_tot);
    // the cut's flags and its count of nodes in skipped tiles
    CK(cudaMemsetAsync(P<uint32_t>(ctx->counters) + C_CUTFLAGS, 0, 2 * sizeof(uint32_t), ctx->stream), "memset");
    w.skipped_nodes = P<uint32_t>(ctx->counters) + C_CUTSKIP;
    bool traverse = n_cams == 1 && ctx->cut_mode == 2;
    if (traverse && ctx->tr_grid < 0) ctx->tr_grid = cut_traverse_grid(ctx->num_sms);
    if (traverse && ctx->tr_grid <= 0) traverse = false;   // no cooperative launch: the scan
    TravArgs ta{};
    if (traverse) {
        const size_t words = (size_t)((N + 31) / 32);
        CK(ensure(ctx->tr_front0, sizeof(uint32_t) * (size_t)N), "traversal frontier");
        CK(ensure(ctx->tr_front1, sizeof(uint32_t) * (size_t)N), "traversal frontier");
        CK(ensure(ctx->tr_feps0, sizeof(float) * (size_t)N), "traversal frontier");
        CK(ensure(ctx->tr_feps1, sizeof(float) * (size_t)N), "traversal frontier");
        CK(ensure(ctx->tr_level, sizeof(uint32_t) * TR_LEVEL_WORDS), "traversal levels");
        CK(ensure(ctx->tr_tnode, sizeof(float) * (size_t)N), "traversal weights");
        CK(ensure(ctx->tr_mark, sizeof(uint32_t) * words), "traversal marks");
        if (ctx->tr_mark_bytes != ctx->tr_mark.n) {   // a new mark buffer: zero it once (each compaction clears it)
            CK(cudaMemsetAsync(ctx->tr_mark.p, 0, ctx->tr_mark.n, ctx->stream), "memset");
            ctx->tr_mark_bytes = ctx->tr_mark.n;
        }
        const int64_t tw = (int64_t)cut_traverse_work_words(N);
        if (tw > w.lb_words) {
            w.lb_words = tw;
            CK(ensure(ctx->cut_lb, sizeof(uint32_t) * (size_t)w.lb_words), "cut look-back");
            w.lb_work = P<uint32_t>(ctx->cut_lb);
        }
        ta.rec = P<const float4>(ctx->rec);
        ta.child_start = ctx->hier.child_start;
        ta.n = N;
        ta.front[0] = P<uint32_t>(ctx->tr_front0);
        ta.front[1] = P<uint32_t>(ctx->tr_front1);
        ta.feps[0] = P<float>(ctx->tr_feps0);
        ta.feps[1] = P<float>(ctx->tr_feps1);
        ta.cap = N;
        ta.level_count = P<uint32_t>(ctx->tr_level);
        ta.inner = ta.level_count + TR_MAX_LEVELS + 1;
        ta.bar = ta.level_count + TR_MAX_LEVELS + 2;
        ta.mark = P<uint32_t>(ctx->tr_mark);
        ta.tnode = P<float>(ctx->tr_tnode);
        ta.flags = P<uint32_t>(ctx->counters) + C_CUTFLAGS;
    }
    stage_begin(ctx, H3DGS_STAGE_CUT);
    if (traverse)
        CK(launch_cut_traverse(ta, cams[0], ctx->tr_grid, w.lb_work, w.lb_words, cut_ids, cut_t, cut_offsets,
                               w.cam_totals, capacity, ctx->stream),
           "traversal cut kernels");
    else
        CK(launch_cut(dev_hier(ctx), P<DevCam>(ctx->cams), n_cams, w, cut_ids, cut_t, cut_offsets, capacity,
                      P<uint32_t>(ctx->counters) + C_CUTFLAGS, ctx->stream),
           "cut kernels");
    stage_end(ctx, H3DGS_STAGE_CUT);
    ctx->last_cut_traversed = traverse;
    if (total_out) {
        int64_t tot = 0;
        CK(cudaMemcpyAsync(&tot, P<int64_t>(ctx->cut_tot) + n_cams, sizeof(int64_t), cudaMemcpyDeviceToHost, ctx->stream),
           "read cut total");
        CK(cudaStreamSynchronize(ctx->stream), "select_cut sync");
        *total_out = tot;
        if (tot > capacity) return fail(ctx, H3DGS_ERR_CAPACITY, "select_cut: cut larger than capacity");
    }
    return H3DGS_OK;
}

h3dgs_status h3dgs_interpolate(h3dgs_ctx* ctx, const h3dgs_camera* cams, int32_t n_cams, const int32_t* cut_ids,
                               const float* cut_t, const int64_t* cut_offsets, int32_t interpolate, float* out,
                               int64_t m_total) {
    if (!ctx) return H3DGS_ERR_INVALID_ARG;
    ctx->err.clear();
    if (!ctx->has_hier) return fail(ctx, H3DGS_ERR_STATE, "interpolate: no hierarchy uploaded");
    h3dgs_status st = check_cams(ctx, cams, n_cams);
    if (st != H3DGS_OK) return st;
    if (m_total < 0 || (m_total > 0 && (!cut_ids || !out)) || !cut_offsets)
        return fail(ctx, H3DGS_ERR_INVALID_ARG, "interpolate: bad outputs");
    if (m_total == 0) return H3DGS_OK;
    CK(cudaSetDevice(ctx->device), "set device");
    CK(launch_interpolate_export(dev_hier(ctx), n_cams, cut_ids, cut_t, cut_offsets, interpolate, out, m_total,
                                 ctx->stream),
       "interpolate");
    return H3DGS_OK;
}

h3dgs_status h3dgs_render(h3dgs_ctx* ctx, const h3dgs_camera* cams, int32_t n_cams, const int32_t* cut_ids,
                          const float* cut_t, const int64_t* cut_offsets, const h3dgs_render_opts* opts, float* images,
                          int32_t save_for_backward) {
    return h3dgs_render_ex(ctx, cams, n_cams, cut_ids, cut_t, cut_offsets, opts, images, nullptr, nullptr,
                           save_for_backward);
}

h3dgs_status h3dgs_render_ex(h3dgs_ctx* ctx, const h3dgs_camera* cams, int32_t n_cams, const int32_t* cut_ids,
                             const float* cut_t, const int64_t* cut_offsets, const h3dgs_render_opts* opts,
                             float* images, float* depth, const float* exposure, int32_t save_for_backward) {
    if (!ctx) return H3DGS_ERR_INVALID_ARG;
    ctx->err.clear();
    if (!ctx->has_hier) return fail(ctx, H3DGS_ERR_STATE, "render: no hierarchy uploaded");
    h3dgs_status st = check_cams(ctx, cams, n_cams);
    if (st != H3DGS_OK) return st;
    if (!opts || !images || !cut_offsets || !cut_ids) return fail(ctx, H3DGS_ERR_INVALID_ARG, "render: NULL argument");
    if (!supported_tile(opts->tile_w, opts->tile_h))
        return fail(ctx, H3DGS_ERR_INVALID_ARG, "render: unsupported tile shape");
    if (!(opts->alpha_clamp > 0 && opts->alpha_clamp < 1) || !(opts->lowpass >= 0) || !(opts->t_min >= 0))
        return fail(ctx, H3DGS_ERR_INVALID_ARG, "render: bad opts");
    if (opts->blend_chunk != 0 && (opts->blend_chunk < 64 || opts->blend_chunk > 65536))
        return fail(ctx, H3DGS_ERR_INVALID_ARG, "render: blend_chunk out of range");
    if ((reinterpret_cast<uintptr_t>(exposure) & 3u) || (reinterpret_cast<uintptr_t>(depth) & 3u))
        return fail(ctx, H3DGS_ERR_INVALID_ARG, "render: misaligned depth or exposure array");
    CK(cudaSetDevice(ctx->device), "set device");
    // with fixed capacities the frame's reset launch also sets up a single batch of cameras
    CamBatch deferred;
    deferred.count = 0;
    st = setup_cameras(ctx, cams, n_cams, opts->tile_w, opts->tile_h, ctx->fixed ? &deferred : nullptr);
    if (st != H3DGS_OK) return st;
    if (ctx->n_tiles > 0xffffffffLL) return fail(ctx, H3DGS_ERR_INVALID_ARG, "render: too many tiles");
    cudaStream_t s = ctx->stream;
    uint32_t* cnt = P<uint32_t>(ctx->counters);
    // ---- capacities
    int64_t capM, capP;
    if (ctx->fixed) {
        capM = ctx->cap_splats;
        capP = ctx->cap_pairs;
    } else {
        int64_t m = 0;
        CK(cudaMemcpyAsync(&m, cut_offsets + n_cams, sizeof(int64_t), cudaMemcpyDeviceToHost, s), "read cut size");
        CK(cudaStreamSynchronize(s), "render sync");
        if (m < 0 || m > 0x7fffffffLL) return fail(ctx, H3DGS_ERR_INVALID_ARG, "render: bad cut size");
        capM = std::max<int64_t>(m, 1);
        const size_t M = (size_t)capM;
        CK(ensure(ctx->s_rec, 16 * SPLAT_F4 * M), "splat buffer");
        CK(ensure(ctx->s_rect, 8 * M), "splat buffer");
        DBuf* m4[] = {&ctx->s_key, &ctx->s_idx, &ctx->s_key2, &ctx->s_idx2, &ctx->s_key3, &ctx->s_tiles,
                      &ctx->s_poff};
        for (DBuf* b : m4) CK(ensure(*b, 4 * M), "splat buffer");
        capP = 0;
    }
    CK(ensure(ctx->ranges, sizeof(int2) * (size_t)ctx->n_tiles), "ranges");
    CK(ensure(ctx->T_final, sizeof(float) * (size_t)ctx->n_pixels), "pixel state");
    CK(ensure(ctx->n_contrib, sizeof(int32_t) * (size_t)ctx->n_pixels), "pixel state");
    // Per-frame clears.  With fixed capacities every workspace the frame clears (the sorts' and scans'
    // look-back words, the blend queue's counters, the digit histograms) has its own region of one
    // buffer, and a single launch clears them with the counters and the tile ranges; otherwise (sizes
    // found on the way) they are cleared where they are used.
    const bool prezero = ctx->fixed;
    uint32_t *depth_hist, *tile_hist, *plan_work = nullptr, *qsync = nullptr;
    SortWork sw_d, sw_t, sw_po;
    size_t plan_words = 0;
    if (prezero) {
        auto r64 = [](size_t w) { return (w + 63) / 64 * 64; };
        const size_t wd = r64(radix_work_words(capM)), wt = r64(radix_work_words(capP));
        const size_t wpo = r64(pair_offsets_work_words(capM)), wpl = r64(blend_plan_work_words(ctx->n_tiles));
        const size_t wq = r64(2 * (size_t)ctx->n_tiles + 1), wh = 2 * 4 * 256;
        const size_t total = wd + wt + wpo + wpl + wq + wh;
        CK(ensure(ctx->fw, sizeof(uint32_t) * total), "frame workspace");
        uint32_t* base = P<uint32_t>(ctx->fw);
        uint32_t* flags = cnt + C_FLAGS;
        sw_d = SortWork{base, wd, ctx->num_sms, flags};
        sw_t = SortWork{base + wd, wt, ctx->num_sms, flags};
        sw_po = SortWork{base + wd + wt, wpo, ctx->num_sms, flags};
        plan_work = base + wd + wt + wpo;
        plan_words = wpl;
        qsync = plan_work + wpl;
        depth_hist = qsync + wq;
        tile_hist = depth_hist + 4 * 256;
        ResetList rl;
        rl.n = 5;
        rl.p[0] = cnt + C_FLAGS;    rl.words[0] = 1;
        rl.p[1] = cnt + C_NVISIBLE; rl.words[1] = 1;
        rl.p[2] = cnt + C_EVALS;    rl.words[2] = EVAL_WORDS;
        rl.p[3] = P<uint32_t>(ctx->ranges); rl.words[3] = 2 * (uint64_t)ctx->n_tiles;
        rl.p[4] = base;             rl.words[4] = total;
        if (deferred.count > 0) {
            rl.cams = P<DevCam>(ctx->cams);
            rl.cb = deferred;
        }
        CK(launch_reset(rl, ctx->num_sms, s), "frame reset");
    } else {
        CK(cudaMemsetAsync(cnt + C_FLAGS, 0, sizeof(uint32_t), s), "memset");
        CK(cudaMemsetAsync(cnt + C_NVISIBLE, 0, sizeof(uint32_t), s), "memset");
        CK(cudaMemsetAsync(cnt + C_EVALS, 0, EVAL_WORDS * sizeof(uint32_t), s), "memset");
        CK(cudaMemsetAsync(ctx->ranges.p, 0, sizeof(int2) * (size_t)ctx->n_tiles, s), "memset");
        CK(ensure(ctx->hists, sizeof(uint32_t) * 2 * 4 * 256), "histograms");
        CK(cudaMemsetAsync(ctx->hists.p, 0, sizeof(uint32_t) * 2 * 4 * 256, s), "memset");
        depth_hist = P<uint32_t>(ctx->hists);
        tile_hist = depth_hist + 4 * 256;
    }
    const DevOpts o = dev_opts(*opts);
    SplatBufs sb;
    sb.rec = P<float4>(ctx->s_rec);
    sb.rect = P<uint2>(ctx->s_rect);
    sb.depth_key = P<uint32_t>(ctx->s_key);
    sb.tiles = P<uint32_t>(ctx->s_tiles);
    sb.n_splats = cnt + C_NSPLATS;
    sb.n_visible = cnt + C_NVISIBLE;
    sb.depth_hist = depth_hist;
    const int grid = ctx->num_sms * 8;
    stage_begin(ctx, H3DGS_STAGE_PREPROCESS);
    CK(launch_preprocess(dev_hier(ctx), P<DevCam>(ctx->cams), n_cams, o, cut_ids, cut_t, cut_offsets, capM, sb,
                         cnt + C_FLAGS, grid, s),
       "preprocess");
    stage_end(ctx, H3DGS_STAGE_PREPROCESS);
    // visible splats by depth (culled ones dropped), pair offsets in that order, pairs, stable sort
    // of the pairs by tile id, ranges
    SortWork sw;
    CK(sort_work(ctx, std::max<int64_t>(capM, ctx->fixed ? capP : 0), &sw), "sort workspace");
    if (!prezero) sw_d = sw_t = sw_po = sw;
    bool in_a = false;
    stage_begin(ctx, H3DGS_STAGE_DEPTH_SORT);
    // the histograms and the kept count (the visible splats) come from the preprocess kernel
    CK(radix_sort_pairs(P<uint32_t>(ctx->s_key), nullptr, P<uint32_t>(ctx->s_key2), P<uint32_t>(ctx->s_idx2),
                        P<uint32_t>(ctx->s_key3), P<uint32_t>(ctx->s_idx), cnt + C_NSPLATS, capM, 32, true,
                        cnt + C_NVISIBLE, sw_d, &in_a, s, depth_hist, prezero),
       "depth sort");
    stage_end(ctx, H3DGS_STAGE_DEPTH_SORT);
    const uint32_t* order = in_a ? P<uint32_t>(ctx->s_idx2) : P<uint32_t>(ctx->s_idx);
    stage_begin(ctx, H3DGS_STAGE_DUPLICATE);
    const int64_t seg_cap0 = ctx->fixed ? capP / DUP_SEG + 2 : 0;
    if (ctx->fixed) CK(ensure(ctx->seg_start, sizeof(uint32_t) * (size_t)seg_cap0), "pair segments");
    CK(launch_pair_offsets(P<uint32_t>(ctx->s_tiles), order, cnt + C_NVISIBLE, capM, P<uint32_t>(ctx->s_poff),
                           P<uint32_t>(ctx->seg_start), seg_cap0, cnt + C_NPAIRS, sw_po, s, prezero),
       "pair offsets");
    if (!ctx->fixed) {
        uint32_t pn = 0;
        CK(cudaMemcpyAsync(&pn, cnt + C_NPAIRS, sizeof(uint32_t), cudaMemcpyDeviceToHost, s), "read pairs");
        CK(cudaStreamSynchronize(s), "render sync");
        capP = std::max<int64_t>(pn, 1);
        DBuf* p4[] = {&ctx->pk0, &ctx->pv0, &ctx->pk1, &ctx->pv1};
        for (DBuf* b : p4) CK(ensure(*b, 4 * (size_t)capP), "pair buffer");
        CK(sort_work(ctx, std::max<int64_t>(capM, capP), &sw), "sort workspace");
        sw_d = sw_t = sw_po = sw;
        const int64_t seg_cap = capP / DUP_SEG + 2;
        CK(ensure(ctx->seg_start, sizeof(uint32_t) * (size_t)seg_cap), "pair segments");
        CK(launch_pair_segments(P<uint32_t>(ctx->s_tiles), order, cnt + C_NVISIBLE, P<uint32_t>(ctx->s_poff),
                                P<uint32_t>(ctx->seg_start), seg_cap, grid, s),
           "pair segments");
    }
    int tbits = 1;
    while (tbits < 32 && ((int64_t)1 << tbits) < ctx->n_tiles) ++tbits;
    CK(launch_duplicate(P<DevCam>(ctx->cams), n_cams, cut_offsets, sb, order, cnt + C_NVISIBLE, P<uint32_t>(ctx->s_poff),
                        P<uint32_t>(ctx->seg_start), cnt + C_NPAIRS, capP, cnt + C_NPAIRS_KEPT, P<uint32_t>(ctx->pk0),
                        P<uint32_t>(ctx->pv0), tile_hist, (tbits + 7) / 8, cnt + C_FLAGS, s),
       "duplicate");
    stage_end(ctx, H3DGS_STAGE_DUPLICATE);
    stage_begin(ctx, H3DGS_STAGE_TILE_SORT);
    // histograms counted by the duplication; every pair is kept
    CK(radix_sort_pairs(P<uint32_t>(ctx->pk0), P<uint32_t>(ctx->pv0), P<uint32_t>(ctx->pk1), P<uint32_t>(ctx->pv1),
                        P<uint32_t>(ctx->pk0), P<uint32_t>(ctx->pv0), cnt + C_NPAIRS_KEPT, capP, tbits, false,
                        cnt + C_NPAIRS_KEPT, sw_t, &in_a, s, tile_hist, prezero,
                        reinterpret_cast<uint32_t*>(P<int2>(ctx->ranges)), ctx->n_tiles),
       "tile sort");
    stage_end(ctx, H3DGS_STAGE_TILE_SORT);
    const bool in1 = in_a;   // the tile sort's last pass also marked the tile ranges (decoded by the plan)
    stage_begin(ctx, H3DGS_STAGE_BLEND);
    {
        const int NT = o.tile_w * o.tile_h;
        const int64_t icap = ctx->n_tiles + capP / (o.chunk > 0 ? o.chunk : BLEND_AUTO_CHUNK) + 1;
        CK(ensure(ctx->items, sizeof(int2) * (size_t)icap), "blend items");
        CK(ensure(ctx->q_prod, sizeof(uint32_t) * (size_t)icap), "blend queue");
        CK(ensure(ctx->q_cons, sizeof(uint32_t) * (size_t)icap), "blend queue");
        CK(ensure(ctx->q_single, sizeof(uint32_t) * (size_t)ctx->n_tiles), "blend queue");
        CK(ensure(ctx->queue_sync, sizeof(uint32_t) * (size_t)(2 * ctx->n_tiles + 1)), "blend queue");
        CK(ensure(ctx->tile_item0, sizeof(int32_t) * (size_t)ctx->n_tiles), "blend items");
        CK(ensure(ctx->tile_nch, sizeof(int32_t) * (size_t)ctx->n_tiles), "blend items");
        CK(ensure(ctx->sc_Tc, sizeof(float) * (size_t)icap * NT), "blend scratch");
        CK(ensure(ctx->sc_C, 3 * sizeof(float) * (size_t)icap * NT), "blend scratch");
        CK(ensure(ctx->sc_Tend, sizeof(float) * (size_t)icap * NT), "blend scratch");
        CK(ensure(ctx->sc_last, sizeof(int32_t) * (size_t)icap * NT), "blend scratch");
        if (depth) CK(ensure(ctx->sc_D, sizeof(float) * (size_t)icap * NT), "blend scratch");
        ctx->has_exposure = exposure != nullptr;
        if (exposure) {
            CK(ensure(ctx->exposure, sizeof(float) * 12 * (size_t)n_cams), "exposure");
            CK(cudaMemcpyAsync(ctx->exposure.p, exposure, sizeof(float) * 12 * (size_t)n_cams, cudaMemcpyDeviceToDevice, s),
               "exposure copy");
        }
        ctx->item_cap = icap;
        ctx->opts = o;
        ctx->pairs_in_1 = in1;
        BlendArgs ba = blend_args(ctx, n_cams, images, depth);
        if (!save_for_backward) {   // the adjoint's per-pixel state is not kept
            ba.T_final = nullptr;
            ba.n_contrib = nullptr;
        }
        if (prezero) {
            ba.work = plan_work;
            ba.work_words = plan_words;
            ba.queue_sync = qsync;
            ba.pre_zeroed = true;
        }
        if (ctx->prof) {
            ba.ev_queue = ctx->ev + 2 * H3DGS_STAGE_BLEND_QUEUE;
            ctx->ev_used[H3DGS_STAGE_BLEND_QUEUE] = true;
        }
        CK(launch_blend(ba, s), "blend");
    }
    stage_end(ctx, H3DGS_STAGE_BLEND);
    ctx->rendered = true;
    ctx->saved = save_for_backward != 0;
    ctx->saved_depth = ctx->saved && depth != nullptr;
    ctx->cut_ids = cut_ids;
    ctx->cut_t = cut_t;
    ctx->cut_offsets = cut_offsets;
    ctx->pairs_in_1 = in1;
    ctx->splat_cap_used = capM;
    ctx->pair_cap_used = capP;
    return H3DGS_OK;
}

h3dgs_status h3dgs_render_backward(h3dgs_ctx* ctx, const float* dL, const h3dgs_grads* g, int32_t freeze_leaves) {
    return h3dgs_render_backward_ex(ctx, dL, nullptr, g, freeze_leaves);
}

h3dgs_status h3dgs_render_backward_ex(h3dgs_ctx* ctx, const float* dL, const float* dL_ddepth, const h3dgs_grads* g,
                                      int32_t freeze_leaves) {
    if (!ctx) return H3DGS_ERR_INVALID_ARG;
    ctx->err.clear();
    if (!ctx->saved || !ctx->has_hier) return fail(ctx, H3DGS_ERR_STATE, "render_backward: no saved forward state");
    if (ctx->streamed) return fail(ctx, H3DGS_ERR_STATE, "render_backward: not available for a streamed hierarchy");
    if (dL_ddepth && !ctx->saved_depth)
        return fail(ctx, H3DGS_ERR_STATE, "render_backward: a depth gradient needs a forward that rendered depth");
    if (!dL || !g || !g->mean || !g->scale || !g->rot || !g->opacity || !g->sh)
        return fail(ctx, H3DGS_ERR_INVALID_ARG, "render_backward: NULL argument");
    if (!aligned16(g->rot) || !aligned16(g->sh))
        return fail(ctx, H3DGS_ERR_INVALID_ARG, "render_backward: rot and sh gradients must be 16-byte aligned");
    CK(cudaSetDevice(ctx->device), "set device");
    const int n_cams = (int)ctx->cams_host.size();
    CK(ensure(ctx->splat_grad, sizeof(float) * 12 * (size_t)ctx->splat_cap_used), "splat gradient buffer");
    CK(cudaMemsetAsync(ctx->splat_grad.p, 0, sizeof(float) * 12 * (size_t)ctx->splat_cap_used, ctx->stream), "memset");
    GradBufs gb{g->mean, g->scale, g->rot, g->opacity, g->sh};
    cudaEvent_t* ev = ctx->prof ? ctx->ev + 2 * H3DGS_STAGE_BACKWARD_BLEND : nullptr;
    BlendArgs ba = blend_args(ctx, n_cams, nullptr, nullptr);
    // the splat stage's grid-stride loop on 16 blocks of 128 per SM (four waves of its 4 resident
    // blocks; 8, 32 and 64 per SM measured slower at the 1080p corridor: 0.085, 0.081, 0.083 ms vs 0.079)
    CK(launch_backward(dev_hier(ctx), ba, ctx->cut_ids, ctx->cut_t, ctx->cut_offsets, P<uint2>(ctx->s_rect),
                       P<uint32_t>(ctx->counters) + C_NSPLATS, dL, dL_ddepth, P<float>(ctx->splat_grad), gb,
                       freeze_leaves, ctx->num_sms * 16, ev, ctx->stream),
       "backward");
    if (ctx->prof) ctx->ev_used[H3DGS_STAGE_BACKWARD_BLEND] = ctx->ev_used[H3DGS_STAGE_BACKWARD_SPLAT] = true;
    return H3DGS_OK;
}

h3dgs_status h3dgs_measure_peaks(h3dgs_ctx* ctx, float* fp32_tflops, float* ex2_gops) {
    if (!ctx) return H3DGS_ERR_INVALID_ARG;
    ctx->err.clear();
    if (!fp32_tflops || !ex2_gops) return fail(ctx, H3DGS_ERR_INVALID_ARG, "measure_peaks: NULL output");
    CK(cudaSetDevice(ctx->device), "set device");
    CK(measure_peaks(ctx->num_sms, fp32_tflops, ex2_gops, ctx->stream), "measure peaks");
    return H3DGS_OK;
}

h3dgs_status h3dgs_get_stats(h3dgs_ctx* ctx, h3dgs_stats* out) {
    if (!ctx || !out) return H3DGS_ERR_INVALID_ARG;
    ctx->err.clear();
    CK(cudaSetDevice(ctx->device), "set device");
    uint32_t c[C_COUNT];
    CK(cudaMemcpyAsync(c, ctx->counters.p, sizeof(c), cudaMemcpyDeviceToHost, ctx->stream), "read counters");
    CK(cudaStreamSynchronize(ctx->stream), "stats sync");
    out->n_cut = c[C_NSPLATS];
    out->n_visible = c[C_NVISIBLE];
    out->n_pairs = c[C_NPAIRS_KEPT];
    out->n_tiles = ctx->n_tiles;
    out->n_pixels = ctx->n_pixels;
    out->device_flags = c[C_FLAGS] | c[C_CUTFLAGS];
    uint64_t ev;
    std::memcpy(&ev, c + C_EVALS, sizeof(ev));
    out->n_evals = (int64_t)ev;
    std::memcpy(&ev, c + C_EVALS_T, sizeof(ev));
    out->n_evals_tpass = (int64_t)ev;
    std::memcpy(&ev, c + C_EVALS_I, sizeof(ev));
    out->n_evals_interp = (int64_t)ev;
    std::memcpy(&ev, c + C_CONTRIB, sizeof(ev));
    out->n_contrib = (int64_t)ev;
    std::memcpy(&ev, c + C_CONTRIB_I, sizeof(ev));
    out->n_contrib_interp = (int64_t)ev;
    // the scan reads every record except those of the rows its bound test skipped
    out->n_cut_visited = ctx->has_hier ? ctx->hier.n_nodes - (int64_t)c[C_CUTSKIP] : 0;
    if (ctx->last_cut_traversed) {   // the root, then every level's frontier
        std::vector<uint32_t> lv(TR_MAX_LEVELS + 2);   // frontier sizes, then the inner visits
        CK(cudaMemcpyAsync(lv.data(), ctx->tr_level.p, sizeof(uint32_t) * lv.size(), cudaMemcpyDeviceToHost,
                           ctx->stream), "read levels");
        CK(cudaStreamSynchronize(ctx->stream), "stats sync");
        int64_t v = 1;
        for (size_t l = 1; l < lv.size(); ++l) v += lv[l];
        out->n_cut_visited = v;
    }
    // bounds-check words of a checked build (always zero otherwise); reading clears them
    struct { const char* file; cudaError_t (*read)(uint32_t*, cudaStream_t); } readers[] = {
        {"cut.cu", check_read_cut}, {"preprocess.cu", check_read_preprocess}, {"sort.cu", check_read_sort},
        {"blend.cu", check_read_blend}, {"backward.cu", check_read_backward}};
    for (const auto& r : readers) {
        uint32_t w[2];
        CK(r.read(w, ctx->stream), "read check words");
        if (w[0]) {
            out->device_flags |= FLAG_BOUNDS;
            if (ctx->err.empty())
                ctx->err = std::string("bounds check failed in ") + r.file + " line " + std::to_string(w[1]);
        }
    }
    out->n_items = c[C_NITEMS];
    return H3DGS_OK;
}

h3dgs_status h3dgs_set_profiling(h3dgs_ctx* ctx, int32_t enable) {
    if (!ctx) return H3DGS_ERR_INVALID_ARG;
    ctx->err.clear();
    CK(cudaSetDevice(ctx->device), "set device");
    if (enable && !ctx->ev[0])
        for (auto& e : ctx->ev) CK(cudaEventCreate(&e), "event create");
    ctx->prof = enable != 0;
    ctx->count = enable >= 2;
    for (bool& u : ctx->ev_used) u = false;
    return H3DGS_OK;
}

h3dgs_status h3dgs_get_stage_times(h3dgs_ctx* ctx, float* ms) {
    if (!ctx || !ms) return H3DGS_ERR_INVALID_ARG;
    ctx->err.clear();
    CK(cudaSetDevice(ctx->device), "set device");
    CK(cudaStreamSynchronize(ctx->stream), "profile sync");
    for (int i = 0; i < H3DGS_STAGE_COUNT; ++i) {
        ms[i] = 0.0f;
        if (ctx->ev_used[i]) CK(cudaEventElapsedTime(&ms[i], ctx->ev[2 * i], ctx->ev[2 * i + 1]), "event time");
    }
    return H3DGS_OK;
}

h3dgs_status h3dgs_debug_tile_lists(h3dgs_ctx* ctx, int32_t cam, int32_t* ranges, int32_t* ids, int64_t cap,
                                    int64_t* n_out) {
    if (!ctx) return H3DGS_ERR_INVALID_ARG;
    ctx->err.clear();
    if (!ctx->rendered) return fail(ctx, H3DGS_ERR_STATE, "debug: nothing rendered");
    if (cam < 0 || cam >= (int)ctx->cams_host.size() || !ranges || !n_out)
        return fail(ctx, H3DGS_ERR_INVALID_ARG, "debug: bad camera or NULL output");
    CK(cudaSetDevice(ctx->device), "set device");
    cudaStream_t s = ctx->stream;
    const int64_t nt = (int64_t)ctx->tiles_x[cam] * ctx->tiles_y[cam];
    std::vector<int2> r(nt);
    CK(cudaMemcpyAsync(r.data(), P<int2>(ctx->ranges) + ctx->tile_base[cam], sizeof(int2) * nt, cudaMemcpyDeviceToHost, s),
       "read ranges");
    uint32_t P_kept = 0;
    CK(cudaMemcpyAsync(&P_kept, P<uint32_t>(ctx->counters) + C_NPAIRS_KEPT, 4, cudaMemcpyDeviceToHost, s), "read count");
    CK(cudaStreamSynchronize(s), "debug sync");
    int64_t lo = INT64_MAX, hi = 0;
    for (int64_t i = 0; i < nt; ++i)
        if (r[i].y > r[i].x) { lo = std::min<int64_t>(lo, r[i].x); hi = std::max<int64_t>(hi, r[i].y); }
    if (lo == INT64_MAX) lo = hi = 0;
    const int64_t n = hi - lo;
    *n_out = n;
    for (int64_t i = 0; i < nt; ++i) {
        ranges[2 * i] = r[i].y > r[i].x ? (int32_t)(r[i].x - lo) : 0;
        ranges[2 * i + 1] = r[i].y > r[i].x ? (int32_t)(r[i].y - lo) : 0;
    }
    if (n > cap) return fail(ctx, H3DGS_ERR_CAPACITY, "debug: ids capacity too small");
    if (n == 0) return H3DGS_OK;
    if (!ids) return fail(ctx, H3DGS_ERR_INVALID_ARG, "debug: NULL ids");
    std::vector<uint32_t> splat(n);
    const uint32_t* list = ctx->pairs_in_1 ? P<uint32_t>(ctx->pv1) : P<uint32_t>(ctx->pv0);
    CK(cudaMemcpyAsync(splat.data(), list + lo, 4 * n, cudaMemcpyDeviceToHost, s), "read lists");
    int64_t m = 0;
    CK(cudaMemcpyAsync(&m, ctx->cut_offsets + ctx->cams_host.size(), 8, cudaMemcpyDeviceToHost, s), "read cut size");
    CK(cudaStreamSynchronize(s), "debug sync");
    std::vector<int32_t> cid(std::max<int64_t>(m, 1));
    if (m > 0) CK(cudaMemcpyAsync(cid.data(), ctx->cut_ids, 4 * m, cudaMemcpyDeviceToHost, s), "read cut ids");
    CK(cudaStreamSynchronize(s), "debug sync");
    for (int64_t i = 0; i < n; ++i) ids[i] = splat[i] < (uint32_t)m ? cid[splat[i]] : -1;
    return H3DGS_OK;
}

h3dgs_status h3dgs_debug_splats(h3dgs_ctx* ctx, float* rec, int32_t* rect, float* rgb, int64_t m) {
    if (!ctx) return H3DGS_ERR_INVALID_ARG;
    ctx->err.clear();
    if (!ctx->rendered) return fail(ctx, H3DGS_ERR_STATE, "debug: nothing rendered");
    if (m < 0 || m > ctx->splat_cap_used) return fail(ctx, H3DGS_ERR_INVALID_ARG, "debug: m out of range");
    CK(cudaSetDevice(ctx->device), "set device");
    cudaStream_t s = ctx->stream;
    std::vector<float4> r(SPLAT_F4 * std::max<int64_t>(m, 1));
    std::vector<uint2> rc(std::max<int64_t>(m, 1));
    std::vector<uint32_t> key(std::max<int64_t>(m, 1));
    if (m > 0) {
        CK(cudaMemcpyAsync(r.data(), ctx->s_rec.p, 16 * SPLAT_F4 * m, cudaMemcpyDeviceToHost, s), "read splats");
        CK(cudaMemcpyAsync(rc.data(), ctx->s_rect.p, 8 * m, cudaMemcpyDeviceToHost, s), "read rects");
        CK(cudaMemcpyAsync(key.data(), ctx->s_key.p, 4 * m, cudaMemcpyDeviceToHost, s), "read depth");
    }
    CK(cudaStreamSynchronize(s), "debug sync");
    std::vector<float> depth(std::max<int64_t>(m, 1), 0.0f);
    for (int64_t i = 0; i < m; ++i) std::memcpy(&depth[i], &key[i], 4);
    for (int64_t i = 0; i < m; ++i) {
        const bool culled = rc[i].x == 0xffffffffu;
        const float4 a = r[SPLAT_F4 * i], b = r[SPLAT_F4 * i + 1], c = r[SPLAT_F4 * i + 2];
        if (rec) {
            float* o = rec + 10 * i;
            if (culled) { for (int k = 0; k < 10; ++k) o[k] = 0.0f; }
            else { o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w; o[4] = b.x; o[5] = b.y; o[6] = b.z; o[7] = b.w; o[8] = c.w; o[9] = depth[i]; }
        }
        if (rect) {
            int32_t* q = rect + 4 * i;
            if (culled) { q[0] = q[1] = q[2] = q[3] = -1; }
            else { q[0] = rc[i].x & 0xffff; q[1] = rc[i].x >> 16; q[2] = rc[i].y & 0xffff; q[3] = rc[i].y >> 16; }
        }
        if (rgb) { rgb[3 * i] = culled ? 0.f : c.x; rgb[3 * i + 1] = culled ? 0.f : c.y; rgb[3 * i + 2] = culled ? 0.f : c.z; }
    }
    return H3DGS_OK;
}

h3dgs_status h3dgs_debug_wait_timeout(h3dgs_ctx* ctx, int32_t polls) {
    if (!ctx) return H3DGS_ERR_INVALID_ARG;
    ctx->err.clear();
    if (polls < 1 || polls > (1 << 20)) return fail(ctx, H3DGS_ERR_INVALID_ARG, "debug: polls out of range");
    CK(cudaSetDevice(ctx->device), "set device");
    uint32_t* cnt = P<uint32_t>(ctx->counters);
    CK(cudaMemsetAsync(cnt + C_FLAGS, 0, sizeof(uint32_t), ctx->stream), "memset");
    // the word waited on is one that nothing sets during the call (the render's item counter slot is
    // reused as a zero word: cleared here, read only)
    CK(cudaMemsetAsync(cnt + C_NSORTED, 0, sizeof(uint32_t), ctx->stream), "memset");
    CK(launch_wait_probe(cnt + C_NSORTED, polls, cnt + C_FLAGS, ctx->stream), "wait probe");
    return H3DGS_OK;
}

h3dgs_status h3dgs_debug_pixel_state(h3dgs_ctx* ctx, float* T_final, int32_t* n_contrib, int64_t n_pixels) {
    if (!ctx) return H3DGS_ERR_INVALID_ARG;
    ctx->err.clear();
    if (!ctx->rendered) return fail(ctx, H3DGS_ERR_STATE, "debug: nothing rendered");
    if (n_pixels != ctx->n_pixels) return fail(ctx, H3DGS_ERR_INVALID_ARG, "debug: n_pixels mismatch");
    CK(cudaSetDevice(ctx->device), "set device");
    if (T_final) CK(cudaMemcpyAsync(T_final, ctx->T_final.p, 4 * n_pixels, cudaMemcpyDeviceToHost, ctx->stream), "read T");
    if (n_contrib) CK(cudaMemcpyAsync(n_contrib, ctx->n_contrib.p, 4 * n_pixels, cudaMemcpyDeviceToHost, ctx->stream), "read n");
    CK(cudaStreamSynchronize(ctx->stream), "debug sync");
    return H3DGS_OK;
}

h3dgs_status h3dgs_set_cut_mode(h3dgs_ctx* ctx, int32_t mode) {
    if (!ctx) return H3DGS_ERR_INVALID_ARG;
    ctx->err.clear();
    if (mode < 0 || mode > 2) return fail(ctx, H3DGS_ERR_INVALID_ARG, "set_cut_mode: mode must be 0, 1 or 2");
    ctx->cut_mode = mode;
    return H3DGS_OK;
}

int32_t h3dgs_build_flags(void) {
#ifdef H3DGS_CHECK
    return H3DGS_BUILD_CHECKED;
#else
    return 0;
#endif
}

}  // extern "C"
