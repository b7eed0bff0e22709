// Fused interpolate + project + SH (a3, a4).
//
// One thread per cut entry.  The entry's node n is interpolated with its parent p using the parent
// weight t (Sec. 4.2): a = (1 - t) a_n + t a_p for mean, scale, rotation (then normalised) and SH,
// computed as fmaf(t, a_p, (1 - t) a_n).  The parent's attributes are only read when t != 0,
// which is why leaves cost about twice the bytes of interior cut nodes (Sec. 8.2).
//
// Projection is EWA splatting: Sigma' = J W Sigma W^T J^T with J the Jacobian of the pinhole map
// at the mean (x/z, y/z clamped to 1.3 tan(half fov)).  Sigma' is evaluated as M M^T with
// M = J W R(q) diag(s) (2x3), and det Sigma' as |M_0 x M_1|^2 (Cauchy-Binet), which stays accurate
// for thin splats.  The screen low-pass adds `lowpass` to the diagonal (Sec. 5.1); with
// aa_compensate the opacities are scaled by sqrt(det Sigma' / det Sigma'_f).  The conic is stored
// pre-scaled by -log2(e)/2 so that the blend evaluates G with one ex2.
//
// Everything that decides an integer (culling, radius, tile rectangle, depth key) is evaluated in
// a fixed fp32 order with non-contracting intrinsics; colour is evaluated freely.
#include "internal.cuh"

namespace h3dgs {

namespace {

constexpr float KH = -0.72134752044448170f;  // -0.5 * log2(e)
constexpr float KL = 1.44269504088896341f;   //  log2(e)

// closed forms: sqrt((2l+1)/(4 pi) (l-|m|)!/(l+|m|)!), times sqrt(2) for m != 0
constexpr float SH_C0 = 0.28209479177387814f;   // 1/(2 sqrt(pi))
constexpr float SH_C1 = 0.48860251190291992f;   // sqrt(3/(4 pi))
constexpr float SH_C2A = 1.0925484305920792f;   // sqrt(15/(4 pi))
constexpr float SH_C2B = 0.31539156525252005f;  // sqrt(5/(16 pi))
constexpr float SH_C2C = 0.54627421529603959f;  // sqrt(15/(16 pi))
constexpr float SH_C3A = 0.59004358992664352f;  // sqrt(35/(32 pi))
constexpr float SH_C3B = 2.8906114426405538f;   // sqrt(105/(4 pi))
constexpr float SH_C3C = 0.45704579946446572f;  // sqrt(21/(32 pi))
constexpr float SH_C3D = 0.37317633259011540f;  // sqrt(7/(16 pi))
constexpr float SH_C3E = 1.4453057213202769f;   // sqrt(105/(16 pi))

__device__ __forceinline__ void sh_basis(float x, float y, float z, float Y[16]) {
    const float xx = x * x, yy = y * y, zz = z * z;
    Y[0] = SH_C0;
    Y[1] = -SH_C1 * y; Y[2] = SH_C1 * z; Y[3] = -SH_C1 * x;
    Y[4] = SH_C2A * x * y; Y[5] = -SH_C2A * y * z; Y[6] = SH_C2B * (2.f * zz - xx - yy);
    Y[7] = -SH_C2A * x * z; Y[8] = SH_C2C * (xx - yy);
    Y[9] = -SH_C3A * y * (3.f * xx - yy); Y[10] = SH_C3B * x * y * z;
    Y[11] = -SH_C3C * y * (4.f * zz - xx - yy); Y[12] = SH_C3D * z * (2.f * zz - 3.f * xx - 3.f * yy);
    Y[13] = -SH_C3C * x * (4.f * zz - xx - yy); Y[14] = SH_C3E * z * (xx - yy);
    Y[15] = -SH_C3A * x * (xx - 3.f * yy);
}

__device__ __forceinline__ float lerp_c(float t, float omt, float an, float ap) { return ffma(t, ap, fmul(omt, an)); }

struct Interp {
    float mean[3], scale[3], q[4];
};

// Interpolated geometry in the fixed fp32 order (mean, scale, normalised rotation).
__device__ __forceinline__ Interp interp_geometry(const DevHier& h, int32_t n, int32_t p, bool use_p, float t) {
    Interp r;
    const float omt = fsub(1.0f, t);
    float4 qn = __ldg(h.rot + n);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        r.mean[d] = __ldg(h.mean + 3 * (int64_t)n + d);
        r.scale[d] = __ldg(h.scale + 3 * (int64_t)n + d);
    }
    if (use_p) {
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            r.mean[d] = lerp_c(t, omt, r.mean[d], __ldg(h.mean + 3 * (int64_t)p + d));
            r.scale[d] = lerp_c(t, omt, r.scale[d], __ldg(h.scale + 3 * (int64_t)p + d));
        }
        const float4 qp = __ldg(h.rot + p);
        qn = make_float4(lerp_c(t, omt, qn.x, qp.x), lerp_c(t, omt, qn.y, qp.y), lerp_c(t, omt, qn.z, qp.z),
                         lerp_c(t, omt, qn.w, qp.w));
    }
    float n2 = fmul(qn.x, qn.x);
    n2 = ffma(qn.y, qn.y, n2);
    n2 = ffma(qn.z, qn.z, n2);
    n2 = ffma(qn.w, qn.w, n2);
    if (n2 > 0.0f) {
        const float nr = fsqrt(n2);
        r.q[0] = fdiv(qn.x, nr); r.q[1] = fdiv(qn.y, nr); r.q[2] = fdiv(qn.z, nr); r.q[3] = fdiv(qn.w, nr);
    } else {
        r.q[0] = 1.0f; r.q[1] = r.q[2] = r.q[3] = 0.0f;
    }
    return r;
}

}  // namespace

__global__ void __launch_bounds__(256) preprocess_kernel(DevHier h, const DevCam* __restrict__ cams, int n_cams,
                                                         DevOpts o, const int32_t* __restrict__ cut_ids,
                                                         const float* __restrict__ cut_t,
                                                         const int64_t* __restrict__ cut_offsets, int64_t cap,
                                                         SplatBufs sb, uint32_t* __restrict__ flags) {
    griddep_launch_dependents();
    griddep_wait();
    __shared__ uint32_t s_hist[4][256];   // digit histograms of the depth keys, for the depth sort
    if (sb.depth_hist) {
        for (int i = threadIdx.x; i < 4 * 256; i += blockDim.x) (&s_hist[0][0])[i] = 0;
        __syncthreads();
    }
    const int64_t m_raw = cut_offsets[n_cams];
    const int64_t M = m_raw < cap ? m_raw : cap;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *sb.n_splats = (uint32_t)M;
        if (m_raw > cap) atomicOr(flags, FLAG_SPLATS_OVERFLOW);
    }
    uint32_t visible = 0;
    for (int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; m < M; m += (int64_t)gridDim.x * blockDim.x) {
        const int k = find_cam(cut_offsets, n_cams, m);
        const DevCam& cam = cams[k];
        const int32_t n = __ldg(cut_ids + m);
        if (!H3DGS_IN(n, h.n)) {   // checked build only: a cut id outside the hierarchy
            sb.tiles[m] = 0;
            sb.depth_key[m] = 0xffffffffu;
            sb.rect[m] = make_uint2(0xffffffffu, 0xffffffffu);
            continue;
        }
        const float t = (o.interpolate && cut_t) ? __ldg(cut_t + m) : 0.0f;
        const int32_t p = __ldg(h.parent + n);
        const bool use_p = (t != 0.0f) && p >= 0 && H3DGS_IN(p, h.n);
        // attribute rows: the node ids, or the cache slots of a streamed hierarchy
        const int32_t rn = h.row_of ? __ldg(h.row_of + n) : n;
        const int32_t rp = (h.row_of && use_p) ? __ldg(h.row_of + p) : p;
        if (rn < 0 || (use_p && rp < 0)) {   // not resident: flagged, left out of the frame
            atomicOr(flags, FLAG_NOT_RESIDENT);
            sb.tiles[m] = 0;
            sb.depth_key[m] = 0xffffffffu;
            sb.rect[m] = make_uint2(0xffffffffu, 0xffffffffu);
            continue;
        }
        // ---- view transform: the node's and the parent's means are transformed separately (compensated)
        // and interpolated in camera space, which equals transforming the interpolated mean but keeps
        // the precision that a lerp of km-scale world coordinates would lose
        const float* W = cam.R;
        float xc[3];
        view_point(W, cam.T, __ldg(h.mean + 3 * (int64_t)rn), __ldg(h.mean + 3 * (int64_t)rn + 1),
                   __ldg(h.mean + 3 * (int64_t)rn + 2), xc);
        if (use_p) {
            float xp[3];
            view_point(W, cam.T, __ldg(h.mean + 3 * (int64_t)rp), __ldg(h.mean + 3 * (int64_t)rp + 1),
                       __ldg(h.mean + 3 * (int64_t)rp + 2), xp);
            const float omt_v = fsub(1.0f, t);
#pragma unroll
            for (int i = 0; i < 3; ++i) xc[i] = lerp_c(t, omt_v, xc[i], xp[i]);
        }
        const float z = xc[2];
        bool vis = z > cam.znear;
        float u = 0, v = 0, ca = 0, cb = 0, cc = 0, comp = 0, sxx = 0, syy = 0;
        int rx0 = 0, rx1 = -1, ry0 = 0, ry1 = -1;
        if (vis) {
            // scale and rotation only for entries in front of the near plane (half the surroundings of a
            // street or city view lie behind the camera)
            const Interp a = interp_geometry(h, rn, rp, use_p, t);
            const float xz = fdiv(xc[0], z), yz = fdiv(xc[1], z);
            u = ffma(cam.fx, xz, cam.cx);
            v = ffma(cam.fy, yz, cam.cy);
            const float txc = fminf(fmaxf(xz, -cam.limx), cam.limx);
            const float tyc = fminf(fmaxf(yz, -cam.limy), cam.limy);
            const float j00 = fdiv(cam.fx, z), j11 = fdiv(cam.fy, z);
            const float j02 = -fmul(j00, txc), j12 = -fmul(j11, tyc);
            const float qw = a.q[0], qx = a.q[1], qy = a.q[2], qz = a.q[3];
            const float xx = fmul(qx, qx), yy = fmul(qy, qy), zz = fmul(qz, qz);
            const float xy = fmul(qx, qy), xz2 = fmul(qx, qz), yz2 = fmul(qy, qz);
            const float wx = fmul(qw, qx), wy = fmul(qw, qy), wz = fmul(qw, qz);
            float Rq[3][3];
            Rq[0][0] = fsub(1.0f, fmul(2.0f, fadd(yy, zz)));
            Rq[0][1] = fmul(2.0f, fsub(xy, wz));
            Rq[0][2] = fmul(2.0f, fadd(xz2, wy));
            Rq[1][0] = fmul(2.0f, fadd(xy, wz));
            Rq[1][1] = fsub(1.0f, fmul(2.0f, fadd(xx, zz)));
            Rq[1][2] = fmul(2.0f, fsub(yz2, wx));
            Rq[2][0] = fmul(2.0f, fsub(xz2, wy));
            Rq[2][1] = fmul(2.0f, fadd(yz2, wx));
            Rq[2][2] = fsub(1.0f, fmul(2.0f, fadd(xx, yy)));
            float A2[2][3];
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                A2[0][j] = ffma(j02, W[6 + j], fmul(j00, W[0 + j]));
                A2[1][j] = ffma(j12, W[6 + j], fmul(j11, W[3 + j]));
            }
            float M[2][3];
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int kk = 0; kk < 3; ++kk) {
                    float acc = fmul(A2[i][0], Rq[0][kk]);
                    acc = ffma(A2[i][1], Rq[1][kk], acc);
                    acc = ffma(A2[i][2], Rq[2][kk], acc);
                    M[i][kk] = fmul(acc, a.scale[kk]);
                }
            float ca2 = fmul(M[0][0], M[0][0]);
            ca2 = ffma(M[0][1], M[0][1], ca2);
            ca2 = ffma(M[0][2], M[0][2], ca2);
            float cc2 = fmul(M[1][0], M[1][0]);
            cc2 = ffma(M[1][1], M[1][1], cc2);
            cc2 = ffma(M[1][2], M[1][2], cc2);
            float cb2 = fmul(M[0][0], M[1][0]);
            cb2 = ffma(M[0][1], M[1][1], cb2);
            cb2 = ffma(M[0][2], M[1][2], cb2);
            const float k0 = ffma(M[0][1], M[1][2], -fmul(M[0][2], M[1][1]));
            const float k1 = ffma(M[0][2], M[1][0], -fmul(M[0][0], M[1][2]));
            const float k2 = ffma(M[0][0], M[1][1], -fmul(M[0][1], M[1][0]));
            float det = fmul(k0, k0);
            det = ffma(k1, k1, det);
            det = ffma(k2, k2, det);
            const float lp = o.lowpass;
            const float af = fadd(ca2, lp), cf = fadd(cc2, lp);
            const float detf = ffma(lp, fadd(fadd(ca2, cc2), lp), det);
            vis = detf > 0.0f;
            sxx = af;
            syy = cf;
            if (vis) {
                comp = o.aa_compensate ? fsqrt(fmaxf(0.0f, fdiv(det, detf))) : 1.0f;
                ca = fmul(fdiv(cf, detf), KH);
                cc = fmul(fdiv(af, detf), KH);
                cb = fmul(fdiv(cb2, detf), KL);
                const float hm = fmul(0.5f, fadd(af, cf));
                const float hd = fmul(0.5f, fsub(af, cf));
                const float disc = fsqrt(ffma(hd, hd, fmul(cb2, cb2)));
                const float lmax = fadd(hm, disc);
                const float r = ceilf(fmul(3.0f, fsqrt(lmax)));
                const float fx0 = floorf(fdiv(fsub(u, r), (float)o.tile_w));
                const float fx1 = floorf(fdiv(fadd(u, r), (float)o.tile_w));
                const float fy0 = floorf(fdiv(fsub(v, r), (float)o.tile_h));
                const float fy1 = floorf(fdiv(fadd(v, r), (float)o.tile_h));
                const float TXm1 = (float)(cam.tiles_x - 1), TYm1 = (float)(cam.tiles_y - 1);
                vis = fx1 >= 0.0f && fx0 <= TXm1 && fy1 >= 0.0f && fy0 <= TYm1;
                if (vis) {
                    rx0 = (int)fmaxf(fx0, 0.0f);
                    rx1 = (int)fminf(fx1, TXm1);
                    ry0 = (int)fmaxf(fy0, 0.0f);
                    ry1 = (int)fminf(fy1, TYm1);
                }
            }
        }
        if (!vis) {
            sb.tiles[m] = 0;
            sb.depth_key[m] = 0xffffffffu;
            sb.rect[m] = make_uint2(0xffffffffu, 0xffffffffu);
            continue;
        }
        ++visible;
        // ---- view-dependent colour (value only), SH interpolated with the same weight
        const float omt = fsub(1.0f, t);
        // direction from the camera centre to the (interpolated) mean: node and parent directions
        // against the compensated centre, interpolated at metre scale
        float dir[3];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const float dn = (__ldg(h.mean + 3 * (int64_t)rn + j) - cam.ch[j]) - cam.cl[j];
            dir[j] = use_p ? lerp_c(t, omt, dn, (__ldg(h.mean + 3 * (int64_t)rp + j) - cam.ch[j]) - cam.cl[j]) : dn;
        }
        float dx = dir[0], dy = dir[1], dz = dir[2];
        const float inv = rsqrtf(dx * dx + dy * dy + dz * dz);
        dx *= inv; dy *= inv; dz *= inv;
        float Y[16];
        sh_basis(dx, dy, dz, Y);
        float rgb[3] = {0.5f, 0.5f, 0.5f};
        const float4* shn = h.sh + 12 * (int64_t)rn;
        const float4* shp = h.sh + 12 * (int64_t)(use_p ? rp : rn);
#pragma unroll
        for (int j = 0; j < 12; ++j) {
            float4 s4 = __ldg(shn + j);
            if (use_p) {
                const float4 q4 = __ldg(shp + j);
                s4 = make_float4(lerp_c(t, omt, s4.x, q4.x), lerp_c(t, omt, s4.y, q4.y), lerp_c(t, omt, s4.z, q4.z),
                                 lerp_c(t, omt, s4.w, q4.w));
            }
            const float sv[4] = {s4.x, s4.y, s4.z, s4.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int c = 4 * j + e;  // coefficient index = k*3 + ch
                rgb[c % 3] = fmaf(sv[e], Y[c / 3], rgb[c % 3]);
            }
        }
        const float on = fmul(__ldg(h.opacity + rn), comp);
        const float op = use_p ? fmul(__ldg(h.opacity + rp), comp) : 0.0f;
        const float K = use_p ? (float)__ldg(h.child_count + p) : 1.0f;
        // alpha-floor box: alpha <= o_max G, and o_max G >= floor only inside the ellipse
        // d^T Sigma'_f^-1 d <= 2 ln(o_max / floor), whose bounding box has half-widths
        // sqrt(2 ln(o_max / floor) Sigma'_f,xx) and likewise in y; inflated by 1% + 0.01 px
        // in the blend's log2 units the same level set is -p2 = log2(o_max / floor) = r2 log2(e) / 2
        const float omax = fmaxf(on, op);
        float hx = -1.0f, hy = -1.0f, rz = -1.0f;
        if (omax > o.alpha_floor) {
            const float r2 = 2.0f * logf(omax / o.alpha_floor);
            hx = sqrtf(r2 * sxx) * 1.01f + 0.01f;
            hy = sqrtf(r2 * syy) * 1.01f + 0.01f;
            rz = r2 * (0.5f * 1.44269504f) * 1.02f + 0.02f;
        }
        sb.rec[SPLAT_F4 * m + 0] = make_float4(u, v, ca, cb);
        sb.rec[SPLAT_F4 * m + 1] = make_float4(cc, on, op, t);
        sb.rec[SPLAT_F4 * m + 2] = make_float4(fmaxf(rgb[0], 0.0f), fmaxf(rgb[1], 0.0f), fmaxf(rgb[2], 0.0f), K);
        sb.rec[SPLAT_F4 * m + 3] = make_float4(hx, hy, rz, z);
        sb.rect[m] = make_uint2((uint32_t)rx0 | ((uint32_t)rx1 << 16), (uint32_t)ry0 | ((uint32_t)ry1 << 16));
        const uint32_t key = __float_as_uint(z);
        sb.depth_key[m] = key;
        sb.tiles[m] = (uint32_t)((rx1 - rx0 + 1) * (ry1 - ry0 + 1));
        if (sb.depth_hist) {
#pragma unroll
            for (int q = 0; q < 4; ++q) atomicAdd(&s_hist[q][(key >> (8 * q)) & 255u], 1u);
        }
    }
    // block-reduce the visible count
    for (int off = 16; off > 0; off >>= 1) visible += __shfl_down_sync(0xffffffffu, visible, off);
    if ((threadIdx.x & 31) == 0 && visible) atomicAdd(sb.n_visible, visible);
    if (sb.depth_hist) {
        __syncthreads();
        for (int i = threadIdx.x; i < 4 * 256; i += blockDim.x) {
            const uint32_t c = (&s_hist[0][0])[i];
            if (c) atomicAdd(sb.depth_hist + i, c);
        }
    }
}

cudaError_t launch_preprocess(const DevHier& h, const DevCam* cams, int n_cams, const DevOpts& o,
                              const int32_t* cut_ids, const float* cut_t, const int64_t* cut_offsets, int64_t cap,
                              const SplatBufs& sb, uint32_t* flags, int grid, cudaStream_t s) {
    return launch_dependent(preprocess_kernel, dim3(grid), dim3(256), s, h, cams, n_cams, o, cut_ids, cut_t, cut_offsets,
                            cap, sb, flags);
}

// ---------------------------------------------------------------------------------- export (a3)

__global__ void __launch_bounds__(256) interpolate_export_kernel(DevHier h, int n_cams, const int32_t* __restrict__ cut_ids,
                                                                 const float* __restrict__ cut_t,
                                                                 const int64_t* __restrict__ cut_offsets, int interpolate,
                                                                 float* __restrict__ out, int64_t m_total) {
    const int64_t M = min(m_total, cut_offsets[n_cams]);
    for (int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; m < M; m += (int64_t)gridDim.x * blockDim.x) {
        const int32_t n = cut_ids[m];
        const float t = (interpolate && cut_t) ? cut_t[m] : 0.0f;
        const int32_t p = h.parent[n];
        const bool use_p = (t != 0.0f) && p >= 0;
        const int32_t rn = h.row_of ? h.row_of[n] : n;
        const int32_t rp = (h.row_of && use_p) ? h.row_of[p] : p;
        if (rn < 0 || (use_p && rp < 0)) {   // not resident
            for (int r = 0; r < NINTERP; ++r) out[(int64_t)r * m_total + m] = __int_as_float(0x7fc00000);
            continue;
        }
        const Interp a = interp_geometry(h, rn, rp, use_p, t);
        for (int d = 0; d < 3; ++d) {
            out[(int64_t)d * m_total + m] = a.mean[d];
            out[(int64_t)(3 + d) * m_total + m] = a.scale[d];
        }
        for (int d = 0; d < 4; ++d) out[(int64_t)(6 + d) * m_total + m] = a.q[d];
        const float omt = fsub(1.0f, t);
        const float* shn = reinterpret_cast<const float*>(h.sh) + (int64_t)NSH * rn;
        const float* shp = reinterpret_cast<const float*>(h.sh) + (int64_t)NSH * (use_p ? rp : rn);
        for (int c = 0; c < NSH; ++c)
            out[(int64_t)(10 + c) * m_total + m] = use_p ? lerp_c(t, omt, shn[c], shp[c]) : shn[c];
        out[(int64_t)58 * m_total + m] = h.opacity[rn];
        out[(int64_t)59 * m_total + m] = use_p ? h.opacity[rp] : 0.0f;
        out[(int64_t)60 * m_total + m] = t;
        out[(int64_t)61 * m_total + m] = use_p ? (float)h.child_count[p] : 1.0f;
    }
}

cudaError_t launch_interpolate_export(const DevHier& h, int n_cams, const int32_t* cut_ids, const float* cut_t,
                                      const int64_t* cut_offsets, int interpolate, float* out, int64_t m_total,
                                      cudaStream_t s) {
    int64_t blocks = (m_total + 255) / 256;
    if (blocks < 1) blocks = 1;
    if (blocks > 148 * 32) blocks = 148 * 32;
    interpolate_export_kernel<<<(unsigned)blocks, 256, 0, s>>>(h, n_cams, cut_ids, cut_t, cut_offsets, interpolate,
                                                               out, m_total);
    return cudaGetLastError();
}

H3DGS_CHECK_READER(check_read_preprocess)

}  // namespace h3dgs
