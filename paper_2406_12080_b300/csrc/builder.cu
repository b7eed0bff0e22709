// Hierarchy construction on the device (Sec. 4.1): 3-sigma leaf boxes, top-down binary median
// split on the longest box axis, bottom-up merge of the children (Eq. merge with weights
// w'_i = o_i S_i, SH merged alike, parent opacity = falloff sum(w'_i) / S_p), top-down orientation
// matching (Sec. 4.2), breadth-first numbering.
//
// The tree's SHAPE depends only on the leaf count (a group of n leaves splits into floor(n/2) and
// the rest), so the host lays it out once (integer bookkeeping).  The data-dependent work runs
// level by level on the device:
//   boxes   the box of every group is the union of its leaves' boxes (order-preserving integer
//           atomics, warp-aggregated while the warp's leaves share a group);
//   split   members are ordered by (mean on the group's longest axis, leaf index) with two stable
//           LSD radix sorts over all leaves (float key, then group rank), and the first floor(n/2)
//           of each group go left;
//   merge   fp64, deepest level first; Jacobi eigen-decomposition of the merged covariance;
//   orient  fp64, root first: the child's axes are reinterpreted by the proper signed axis
//           permutation (24 candidates) that minimises its rotation relative to the parent.
#include <algorithm>
#include <cmath>
#include <vector>

#include "internal.cuh"

namespace h3dgs {

namespace {

constexpr int NA = 59;  // mean 3, scale 3, rot 4, opacity 1, sh 48 (fp64 work row)
constexpr double PI_D = 3.14159265358979323846;

__device__ __forceinline__ uint32_t enc_f(float f) {
    const uint32_t b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float dec_f(uint32_t e) {
    return __uint_as_float((e & 0x80000000u) ? (e & 0x7fffffffu) : ~e);
}
// ordered key of a float for the radix sort (ascending order of the floats)
__device__ __forceinline__ uint32_t order_key(float f) { return enc_f(f); }

struct D3 { double a[3][3]; };

// rotation matrix of a quaternion (w, x, y, z), normalised first; fixed op order, no contraction
__device__ D3 rot_of(const double q[4]) {
    double n2 = __dmul_rn(q[0], q[0]);
    n2 = __dadd_rn(n2, __dmul_rn(q[1], q[1]));
    n2 = __dadd_rn(n2, __dmul_rn(q[2], q[2]));
    n2 = __dadd_rn(n2, __dmul_rn(q[3], q[3]));
    const double n = __dsqrt_rn(n2);
    const double w = __ddiv_rn(q[0], n), x = __ddiv_rn(q[1], n), y = __ddiv_rn(q[2], n), z = __ddiv_rn(q[3], n);
    const double xx = __dmul_rn(x, x), yy = __dmul_rn(y, y), zz = __dmul_rn(z, z);
    const double xy = __dmul_rn(x, y), xz = __dmul_rn(x, z), yz = __dmul_rn(y, z);
    const double wx = __dmul_rn(w, x), wy = __dmul_rn(w, y), wz = __dmul_rn(w, z);
    D3 r;
    r.a[0][0] = __dsub_rn(1.0, __dmul_rn(2.0, __dadd_rn(yy, zz)));
    r.a[0][1] = __dmul_rn(2.0, __dsub_rn(xy, wz));
    r.a[0][2] = __dmul_rn(2.0, __dadd_rn(xz, wy));
    r.a[1][0] = __dmul_rn(2.0, __dadd_rn(xy, wz));
    r.a[1][1] = __dsub_rn(1.0, __dmul_rn(2.0, __dadd_rn(xx, zz)));
    r.a[1][2] = __dmul_rn(2.0, __dsub_rn(yz, wx));
    r.a[2][0] = __dmul_rn(2.0, __dsub_rn(xz, wy));
    r.a[2][1] = __dmul_rn(2.0, __dadd_rn(yz, wx));
    r.a[2][2] = __dsub_rn(1.0, __dmul_rn(2.0, __dadd_rn(xx, yy)));
    return r;
}

// quaternion of a rotation matrix (largest-component branch), normalised
__device__ void quat_of(const D3& m, double q[4]) {
    const auto& R = m.a;
    const double tr = R[0][0] + R[1][1] + R[2][2];
    if (tr > 0) {
        const double S = sqrt(tr + 1.0) * 2;
        q[0] = 0.25 * S; q[1] = (R[2][1] - R[1][2]) / S; q[2] = (R[0][2] - R[2][0]) / S; q[3] = (R[1][0] - R[0][1]) / S;
    } else if (R[0][0] > R[1][1] && R[0][0] > R[2][2]) {
        const double S = sqrt(1.0 + R[0][0] - R[1][1] - R[2][2]) * 2;
        q[0] = (R[2][1] - R[1][2]) / S; q[1] = 0.25 * S; q[2] = (R[0][1] + R[1][0]) / S; q[3] = (R[0][2] + R[2][0]) / S;
    } else if (R[1][1] > R[2][2]) {
        const double S = sqrt(1.0 + R[1][1] - R[0][0] - R[2][2]) * 2;
        q[0] = (R[0][2] - R[2][0]) / S; q[1] = (R[0][1] + R[1][0]) / S; q[2] = 0.25 * S; q[3] = (R[1][2] + R[2][1]) / S;
    } else {
        const double S = sqrt(1.0 + R[2][2] - R[0][0] - R[1][1]) * 2;
        q[0] = (R[1][0] - R[0][1]) / S; q[1] = (R[0][2] + R[2][0]) / S; q[2] = (R[1][2] + R[2][1]) / S; q[3] = 0.25 * S;
    }
    const double n = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    for (int i = 0; i < 4; ++i) q[i] /= n;
}

// surface area of an ellipsoid, Knud Thomsen's formula (p = 1.6075)
__device__ double area_of(const double s[3]) {
    const double p = 1.6075;
    const double a = pow(s[0], p), b = pow(s[1], p), c = pow(s[2], p);
    return 4.0 * PI_D * pow((a * b + a * c + b * c) / 3.0, 1.0 / p);
}

// symmetric 3x3 eigen-decomposition by cyclic Jacobi rotations; eigenvectors in the columns of V
__device__ void eigen_sym(D3 A, double lam[3], D3& V) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) V.a[i][j] = (i == j) ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 64; ++sweep) {
        const double off = A.a[0][1] * A.a[0][1] + A.a[0][2] * A.a[0][2] + A.a[1][2] * A.a[1][2];
        const double dg = A.a[0][0] * A.a[0][0] + A.a[1][1] * A.a[1][1] + A.a[2][2] * A.a[2][2];
        if (off == 0.0 || off <= 1e-40 * dg) break;
        for (int p = 0; p < 2; ++p)
            for (int q = p + 1; q < 3; ++q) {
                const double apq = A.a[p][q];
                if (apq == 0.0) continue;
                const double th = (A.a[q][q] - A.a[p][p]) / (2.0 * apq);
                const double t = (th >= 0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
                const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < 3; ++k) {
                    const double x = A.a[k][p], y = A.a[k][q];
                    A.a[k][p] = c * x - s * y;
                    A.a[k][q] = s * x + c * y;
                }
                for (int k = 0; k < 3; ++k) {
                    const double x = A.a[p][k], y = A.a[q][k];
                    A.a[p][k] = c * x - s * y;
                    A.a[q][k] = s * x + c * y;
                }
                for (int k = 0; k < 3; ++k) {
                    const double x = V.a[k][p], y = V.a[k][q];
                    V.a[k][p] = c * x - s * y;
                    V.a[k][q] = s * x + c * y;
                }
            }
    }
    for (int i = 0; i < 3; ++i) lam[i] = A.a[i][i];
}

// ---------------------------------------------------------------------------------------- kernels

__global__ void leaf_init_kernel(int64_t L, const float* __restrict__ mean, const float* __restrict__ scale,
                                 const float* __restrict__ rot, const float* __restrict__ given_box,
                                 float* __restrict__ lbox /*[L][6]*/, int32_t* __restrict__ seg,
                                 uint32_t* __restrict__ perm) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < L; i += (int64_t)gridDim.x * blockDim.x) {
        seg[i] = 0;
        perm[i] = (uint32_t)i;
        if (given_box) {   // explicit leaf boxes (min xyz, max xyz)
            for (int k = 0; k < 6; ++k) lbox[6 * i + k] = given_box[6 * i + k];
            continue;
        }
        const double q[4] = {rot[4 * i], rot[4 * i + 1], rot[4 * i + 2], rot[4 * i + 3]};
        const double s[3] = {scale[3 * i], scale[3 * i + 1], scale[3 * i + 2]};
        const D3 R = rot_of(q);
        for (int j = 0; j < 3; ++j) {
            double v = 0.0;
            for (int k = 0; k < 3; ++k) {
                const double e = __dmul_rn(R.a[j][k], s[k]);
                v = __dadd_rn(v, __dmul_rn(e, e));
            }
            const double h = __dmul_rn(3.0, __dsqrt_rn(v));
            const double m = mean[3 * i + j];
            lbox[6 * i + j] = __double2float_rn(__dsub_rn(m, h));
            lbox[6 * i + 3 + j] = __double2float_rn(__dadd_rn(m, h));
        }
    }
}

// node id of every leaf (inverse of leaf_of_node over the leaf nodes)
__global__ void leaf_node_kernel(int64_t N, const int32_t* __restrict__ child_count,
                                 const int32_t* __restrict__ leaf_of_node, int32_t* __restrict__ leaf_node) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < N; v += (int64_t)gridDim.x * blockDim.x)
        if (child_count[v] == 0) leaf_node[leaf_of_node[v]] = (int32_t)v;
}

__global__ void box_reset_kernel(int64_t n, uint32_t* __restrict__ ebox) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        ebox[6 * i + 0] = ebox[6 * i + 1] = ebox[6 * i + 2] = 0xffffffffu;  // min (encoded)
        ebox[6 * i + 3] = ebox[6 * i + 4] = ebox[6 * i + 5] = 0u;           // max (encoded)
    }
}

// union of member boxes per group (group = internal node at this level, by rank)
__global__ void group_boxes_kernel(int64_t L, const uint32_t* __restrict__ perm, const int32_t* __restrict__ seg,
                                   const float* __restrict__ lbox, const int32_t* __restrict__ level_nodes,
                                   uint32_t* __restrict__ ebox) {
    const int lane = threadIdx.x & 31;
    for (int64_t p0 = blockIdx.x * (int64_t)blockDim.x; p0 < L; p0 += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = p0 + threadIdx.x;
        int32_t s = -1;
        uint32_t e[6] = {0xffffffffu, 0xffffffffu, 0xffffffffu, 0u, 0u, 0u};
        if (p < L) {
            const uint32_t l = perm[p];
            s = seg[l];
            if (s >= 0)
                for (int k = 0; k < 3; ++k) {
                    e[k] = enc_f(lbox[6 * (int64_t)l + k]);
                    e[3 + k] = enc_f(lbox[6 * (int64_t)l + 3 + k]);
                }
        }
        const int32_t s0 = __shfl_sync(0xffffffffu, s, 0);
        const bool uniform = __all_sync(0xffffffffu, s == s0);
        if (uniform) {
            if (s0 < 0) continue;
            for (int off = 16; off > 0; off >>= 1)
                for (int k = 0; k < 3; ++k) {
                    e[k] = min(e[k], __shfl_xor_sync(0xffffffffu, e[k], off));
                    e[3 + k] = max(e[3 + k], __shfl_xor_sync(0xffffffffu, e[3 + k], off));
                }
            if (lane == 0) {
                uint32_t* b = ebox + 6 * (int64_t)level_nodes[s0];
                for (int k = 0; k < 3; ++k) { atomicMin(b + k, e[k]); atomicMax(b + 3 + k, e[3 + k]); }
            }
        } else if (s >= 0) {
            uint32_t* b = ebox + 6 * (int64_t)level_nodes[s];
            for (int k = 0; k < 3; ++k) { atomicMin(b + k, e[k]); atomicMax(b + 3 + k, e[3 + k]); }
        }
    }
}

// longest box axis of each group (extents in fp64 from the fp32 box, ties to the lower axis)
__global__ void group_axis_kernel(int64_t G, const int32_t* __restrict__ level_nodes, const uint32_t* __restrict__ ebox,
                                  int8_t* __restrict__ axis) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < G; r += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t* b = ebox + 6 * (int64_t)level_nodes[r];
        int a = 0;
        double best = (double)dec_f(b[3]) - (double)dec_f(b[0]);
        for (int k = 1; k < 3; ++k) {
            const double e = (double)dec_f(b[3 + k]) - (double)dec_f(b[k]);
            if (e > best) { best = e; a = k; }
        }
        axis[r] = (int8_t)a;
    }
}

// keys in leaf order: low word = ordered mean on the group's axis; value = leaf index
__global__ void split_keys_kernel(int64_t L, const float* __restrict__ mean, const int32_t* __restrict__ seg,
                                  const int8_t* __restrict__ axis, uint32_t* __restrict__ key, uint32_t* __restrict__ val) {
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < L; l += (int64_t)gridDim.x * blockDim.x) {
        const int32_t s = seg[l];
        key[l] = s >= 0 ? order_key(mean[3 * l + axis[s]]) : 0xffffffffu;
        val[l] = (uint32_t)l;
    }
}

// high word (group rank) in the order left by the first sort
__global__ void group_keys_kernel(int64_t L, const int32_t* __restrict__ seg, uint32_t n_groups,
                                  const uint32_t* __restrict__ val, uint32_t* __restrict__ key) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < L; p += (int64_t)gridDim.x * blockDim.x) {
        const int32_t s = seg[val[p]];
        key[p] = s >= 0 ? (uint32_t)s : n_groups;
    }
}

// sorted position p of group s at rank r = p - start(s): first floor(cnt/2) go to the left child
__global__ void assign_kernel(int64_t n_active, const uint32_t* __restrict__ gkey, const uint32_t* __restrict__ val,
                              const int64_t* __restrict__ gstart, const int32_t* __restrict__ gcount,
                              const int32_t* __restrict__ child_next /*[G][2]: next rank or -1-node*/,
                              int32_t* __restrict__ seg, int32_t* __restrict__ leaf_of_node) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n_active; p += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t s = gkey[p];
        const uint32_t l = val[p];
        const int64_t r = p - gstart[s];
        const int side = r < (int64_t)(gcount[s] / 2) ? 0 : 1;
        const int32_t c = child_next[2 * (int64_t)s + side];
        if (c >= 0) {
            seg[l] = c;
        } else {
            seg[l] = -1;
            leaf_of_node[-1 - c] = (int32_t)l;
        }
    }
}

__global__ void leaf_nodes_kernel(int64_t N, const int32_t* __restrict__ child_count, const int32_t* __restrict__ leaf_of_node,
                                  const float* __restrict__ mean, const float* __restrict__ scale,
                                  const float* __restrict__ rot, const float* __restrict__ opacity,
                                  const float* __restrict__ sh, const float* __restrict__ lbox, double* __restrict__ work,
                                  uint32_t* __restrict__ ebox) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < N; v += (int64_t)gridDim.x * blockDim.x) {
        if (child_count[v] != 0) continue;
        const int64_t l = leaf_of_node[v];
        double* w = work + NA * v;
        for (int k = 0; k < 3; ++k) { w[k] = mean[3 * l + k]; w[3 + k] = scale[3 * l + k]; }
        for (int k = 0; k < 4; ++k) w[6 + k] = rot[4 * l + k];
        w[10] = opacity[l];
        for (int c = 0; c < NSH; ++c) w[11 + c] = sh[NSH * l + c];
        for (int k = 0; k < 6; ++k) ebox[6 * v + k] = enc_f(lbox[6 * l + k]);
    }
}

// merge the two children of every internal node of one level
__global__ void merge_kernel(int64_t n, const int32_t* __restrict__ level_nodes, const int32_t* __restrict__ child_start,
                             double* __restrict__ work) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = level_nodes[r];
        const int64_t c0 = child_start[v];
        const double* ch[2] = {work + NA * c0, work + NA * (c0 + 1)};
        double wp[2], W = 0.0;
        for (int i = 0; i < 2; ++i) {
            wp[i] = ch[i][10] * area_of(ch[i] + 3);
            W += wp[i];
        }
        double w[2];
        for (int i = 0; i < 2; ++i) w[i] = W > 0 ? wp[i] / W : 0.5;
        double* out = work + NA * v;
        double mu[3] = {0, 0, 0};
        for (int i = 0; i < 2; ++i)
            for (int d = 0; d < 3; ++d) mu[d] += w[i] * ch[i][d];
        D3 S;
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) S.a[a][b] = 0.0;
        for (int i = 0; i < 2; ++i) {
            const D3 R = rot_of(ch[i] + 6);
            const double* s = ch[i] + 3;
            const double dm[3] = {ch[i][0] - mu[0], ch[i][1] - mu[1], ch[i][2] - mu[2]};
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) {
                    double c = 0.0;
                    for (int k = 0; k < 3; ++k) c += R.a[a][k] * s[k] * s[k] * R.a[b][k];
                    S.a[a][b] += w[i] * (c + dm[a] * dm[b]);
                }
        }
        for (int c = 0; c < NSH; ++c) out[11 + c] = w[0] * ch[0][11 + c] + w[1] * ch[1][11 + c];
        double lam[3];
        D3 V;
        eigen_sym(S, lam, V);
        int o0 = 0, o1 = 1, o2 = 2;  // indices by decreasing eigenvalue
        if (lam[o1] > lam[o0]) { int t = o0; o0 = o1; o1 = t; }
        if (lam[o2] > lam[o1]) { int t = o1; o1 = o2; o2 = t; }
        if (lam[o1] > lam[o0]) { int t = o0; o0 = o1; o1 = t; }
        const int ord[3] = {o0, o1, o2};
        D3 Rm;
        double sc[3];
        for (int j = 0; j < 3; ++j) {
            sc[j] = sqrt(fmax(lam[ord[j]], 0.0));
            for (int i = 0; i < 3; ++i) Rm.a[i][j] = V.a[i][ord[j]];
        }
        const double det = Rm.a[0][0] * (Rm.a[1][1] * Rm.a[2][2] - Rm.a[1][2] * Rm.a[2][1]) -
                           Rm.a[0][1] * (Rm.a[1][0] * Rm.a[2][2] - Rm.a[1][2] * Rm.a[2][0]) +
                           Rm.a[0][2] * (Rm.a[1][0] * Rm.a[2][1] - Rm.a[1][1] * Rm.a[2][0]);
        if (det < 0)
            for (int i = 0; i < 3; ++i) Rm.a[i][2] = -Rm.a[i][2];
        double q[4];
        quat_of(Rm, q);
        for (int d = 0; d < 3; ++d) { out[d] = mu[d]; out[3 + d] = sc[d]; }
        for (int d = 0; d < 4; ++d) out[6 + d] = q[d];
        const double Sp = area_of(sc);
        out[10] = Sp > 0 ? W / Sp : 0.0;
    }
}

// signed axis permutations with det +1, in a fixed order: permutations of (0, 1, 2) in
// lexicographic order, sign patterns in binary order (+ before -)
__constant__ int8_t c_perm[24][3];
__constant__ int8_t c_sign[24][3];

__global__ void orient_kernel(int64_t n, const int32_t* __restrict__ level_nodes, const int32_t* __restrict__ child_start,
                              const int32_t* __restrict__ child_count, double* __restrict__ work, int orient_leaves) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = level_nodes[r];
        const double* par = work + NA * v;
        const D3 Rp = rot_of(par + 6);
        for (int ci = 0; ci < child_count[v]; ++ci) {
            if (!orient_leaves && child_count[(int64_t)child_start[v] + ci] == 0) continue;
            double* ch = work + NA * ((int64_t)child_start[v] + ci);
            const D3 Rc = rot_of(ch + 6);
            int best = 0;
            double best_tr = -1e300;
            for (int k = 0; k < 24; ++k) {
                double tr = 0.0;
                for (int j = 0; j < 3; ++j)
                    for (int i = 0; i < 3; ++i) tr += Rp.a[i][j] * (double)c_sign[k][j] * Rc.a[i][c_perm[k][j]];
                if (tr > best_tr) { best_tr = tr; best = k; }
            }
            D3 Rn;
            double sn[3];
            for (int j = 0; j < 3; ++j) {
                sn[j] = ch[3 + c_perm[best][j]];
                for (int i = 0; i < 3; ++i) Rn.a[i][j] = (double)c_sign[best][j] * Rc.a[i][c_perm[best][j]];
            }
            double q[4];
            quat_of(Rn, q);
            double dot = 0.0;
            for (int i = 0; i < 4; ++i) dot += q[i] * par[6 + i];
            if (dot < 0)
                for (int i = 0; i < 4; ++i) q[i] = -q[i];
            for (int j = 0; j < 3; ++j) ch[3 + j] = sn[j];
            for (int i = 0; i < 4; ++i) ch[6 + i] = q[i];
        }
    }
}

__global__ void output_kernel(int64_t N, const double* __restrict__ work, const uint32_t* __restrict__ ebox,
                              float* __restrict__ mean, float* __restrict__ scale, float* __restrict__ rot,
                              float* __restrict__ opacity, float* __restrict__ sh, float* __restrict__ bmin,
                              float* __restrict__ bmax) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < N; v += (int64_t)gridDim.x * blockDim.x) {
        const double* w = work + NA * v;
        for (int k = 0; k < 3; ++k) {
            mean[3 * v + k] = (float)w[k];
            scale[3 * v + k] = (float)w[3 + k];
            bmin[3 * v + k] = dec_f(ebox[6 * v + k]);
            bmax[3 * v + k] = dec_f(ebox[6 * v + 3 + k]);
        }
        for (int k = 0; k < 4; ++k) rot[4 * v + k] = (float)w[6 + k];
        opacity[v] = (float)w[10];
        for (int c = 0; c < NSH; ++c) sh[NSH * v + c] = (float)w[11 + c];
    }
}

}  // namespace

// --------------------------------------------------------------------------------------- host side

struct BuildShape {
    std::vector<int32_t> parent, child_start, child_count;
    std::vector<int64_t> lo;
    std::vector<int32_t> cnt;
    std::vector<int64_t> level_start;  // node id range of each depth
};

// Breadth-first shape of the median-split tree over L leaves (depends on L only).
static void make_shape(int64_t L, BuildShape& s) {
    const int64_t N = 2 * L - 1;
    s.parent.assign(N, -1);
    s.child_start.assign(N, -1);
    s.child_count.assign(N, 0);
    s.lo.assign(N, 0);
    s.cnt.assign(N, 0);
    s.lo[0] = 0;
    s.cnt[0] = (int32_t)L;
    int64_t next = 1;
    s.level_start = {0};
    int64_t lvl_end = 1;
    for (int64_t v = 0; v < N; ++v) {
        if (v == lvl_end) {
            s.level_start.push_back(v);
            lvl_end = next;
        }
        const int32_t n = s.cnt[v];
        if (n < 2) continue;
        s.child_start[v] = (int32_t)next;
        s.child_count[v] = 2;
        s.lo[next] = s.lo[v];
        s.cnt[next] = n / 2;
        s.lo[next + 1] = s.lo[v] + n / 2;
        s.cnt[next + 1] = n - n / 2;
        s.parent[next] = s.parent[next + 1] = (int32_t)v;
        next += 2;
    }
    s.level_start.push_back(N);
}

namespace {

struct DevMem {
    std::vector<void*> ptrs;
    ~DevMem() {
        for (void* p : ptrs) cudaFree(p);
    }
    template <typename T>
    cudaError_t alloc(T** p, size_t n) {
        cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), std::max<size_t>(n, 1) * sizeof(T));
        if (e == cudaSuccess) ptrs.push_back(*p);
        return e;
    }
};

bool g_perm_ready = false;

cudaError_t upload_perms() {
    if (g_perm_ready) return cudaSuccess;
    int8_t perm[24][3], sign[24][3];
    int k = 0;
    const int P[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
    const int par[6] = {1, -1, -1, 1, 1, -1};
    for (int p = 0; p < 6; ++p)
        for (int bits = 0; bits < 8; ++bits) {
            const int s0 = (bits >> 2) & 1 ? -1 : 1, s1 = (bits >> 1) & 1 ? -1 : 1, s2 = bits & 1 ? -1 : 1;
            if (par[p] * s0 * s1 * s2 > 0) {
                for (int j = 0; j < 3; ++j) perm[k][j] = (int8_t)P[p][j];
                sign[k][0] = (int8_t)s0;
                sign[k][1] = (int8_t)s1;
                sign[k][2] = (int8_t)s2;
                ++k;
            }
        }
    cudaError_t e = cudaMemcpyToSymbol(c_perm, perm, sizeof(perm));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_sign, sign, sizeof(sign));
    if (e == cudaSuccess) g_perm_ready = true;
    return e;
}

}  // namespace

#define BR(x)                                   \
    do {                                        \
        cudaError_t e_ = (x);                   \
        if (e_ != cudaSuccess) return e_;       \
    } while (0)

cudaError_t build_hierarchy(int64_t L, const float* mean, const float* scale, const float* rot, const float* opacity,
                            const float* sh, const BuildOut& out, const SortWork& sw, int num_sms, cudaStream_t st,
                            const BuildExtra& ex) {
    BR(upload_perms());
    const int64_t N = 2 * L - 1;
    BuildShape shape;
    make_shape(L, shape);
    const int n_levels = (int)shape.level_start.size() - 1;
    // per level: internal nodes in rank order
    std::vector<std::vector<int32_t>> lvl_nodes(n_levels);
    std::vector<int32_t> rank_of(N, -1);
    for (int d = 0; d < n_levels; ++d)
        for (int64_t v = shape.level_start[d]; v < shape.level_start[d + 1]; ++v)
            if (shape.cnt[v] >= 2) {
                rank_of[v] = (int32_t)lvl_nodes[d].size();
                lvl_nodes[d].push_back((int32_t)v);
            }
    size_t maxG = 1;
    for (auto& v : lvl_nodes) maxG = std::max(maxG, v.size());
    DevMem mem;
    float* lbox;
    int32_t *seg, *leaf_of_node, *d_nodes, *d_cnt, *d_next;
    uint32_t *perm, *k0, *v0, *k1, *v1, *ebox, *n_dev;
    int64_t* d_start;
    int8_t* d_axis;
    double* work;
    BR(mem.alloc(&lbox, 6 * (size_t)L));
    BR(mem.alloc(&seg, (size_t)L));
    BR(mem.alloc(&leaf_of_node, (size_t)N));
    BR(mem.alloc(&perm, (size_t)L));
    BR(mem.alloc(&k0, (size_t)L));
    BR(mem.alloc(&v0, (size_t)L));
    BR(mem.alloc(&k1, (size_t)L));
    BR(mem.alloc(&v1, (size_t)L));
    BR(mem.alloc(&ebox, 6 * (size_t)N));
    BR(mem.alloc(&n_dev, 2));   // [0] leaf count, [1] kept count of the sorts
    BR(mem.alloc(&d_nodes, maxG));
    BR(mem.alloc(&d_cnt, maxG));
    BR(mem.alloc(&d_next, 2 * maxG));
    BR(mem.alloc(&d_start, maxG));
    BR(mem.alloc(&d_axis, maxG));
    BR(mem.alloc(&work, (size_t)NA * N));
    const int grid = num_sms * 8;
    const uint32_t L32 = (uint32_t)L;
    BR(cudaMemcpyAsync(n_dev, &L32, sizeof(uint32_t), cudaMemcpyHostToDevice, st));
    BR(cudaMemcpyAsync(out.parent, shape.parent.data(), 4 * N, cudaMemcpyHostToDevice, st));
    BR(cudaMemcpyAsync(out.child_start, shape.child_start.data(), 4 * N, cudaMemcpyHostToDevice, st));
    BR(cudaMemcpyAsync(out.child_count, shape.child_count.data(), 4 * N, cudaMemcpyHostToDevice, st));
    leaf_init_kernel<<<grid, 256, 0, st>>>(L, mean, scale, rot, ex.leaf_box, lbox, seg, perm);
    box_reset_kernel<<<grid, 256, 0, st>>>(N, ebox);
    const int32_t zero = 0;
    if (L == 1) BR(cudaMemcpyAsync(leaf_of_node, &zero, 4, cudaMemcpyHostToDevice, st));
    BR(cudaGetLastError());
    std::vector<int32_t> cnt_h, next_h;
    std::vector<int64_t> start_h;
    for (int d = 0; d < n_levels; ++d) {
        const auto& nodes = lvl_nodes[d];
        const int64_t G = (int64_t)nodes.size();
        if (G == 0) continue;
        cnt_h.resize(G);
        start_h.resize(G);
        next_h.resize(2 * G);
        int64_t run = 0;
        for (int64_t r = 0; r < G; ++r) {
            const int32_t v = nodes[r];
            cnt_h[r] = shape.cnt[v];
            start_h[r] = run;
            run += shape.cnt[v];
            for (int c = 0; c < 2; ++c) {
                const int32_t ch = shape.child_start[v] + c;
                next_h[2 * r + c] = shape.cnt[ch] >= 2 ? rank_of[ch] : -1 - ch;
            }
        }
        const int64_t n_active = run;
        BR(cudaMemcpyAsync(d_nodes, nodes.data(), 4 * G, cudaMemcpyHostToDevice, st));
        BR(cudaMemcpyAsync(d_cnt, cnt_h.data(), 4 * G, cudaMemcpyHostToDevice, st));
        BR(cudaMemcpyAsync(d_start, start_h.data(), 8 * G, cudaMemcpyHostToDevice, st));
        BR(cudaMemcpyAsync(d_next, next_h.data(), 8 * G, cudaMemcpyHostToDevice, st));
        group_boxes_kernel<<<grid, 256, 0, st>>>(L, perm, seg, lbox, d_nodes, ebox);
        group_axis_kernel<<<grid, 256, 0, st>>>(G, d_nodes, ebox, d_axis);
        split_keys_kernel<<<grid, 256, 0, st>>>(L, mean, seg, d_axis, k0, v0);
        bool in1 = false;
        BR(radix_sort_pairs(k0, v0, k1, v1, k0, v0, n_dev, L, 32, false, n_dev + 1, sw, &in1, st));
        uint32_t* va = in1 ? v1 : v0;   // leaves in (mean on axis, leaf index) order
        uint32_t* kb = in1 ? k0 : k1;   // free key buffer
        uint32_t* kc = in1 ? k1 : k0;   // keys of the first sort, no longer needed
        uint32_t* vb = in1 ? v0 : v1;   // free value buffer
        group_keys_kernel<<<grid, 256, 0, st>>>(L, seg, (uint32_t)G, va, kb);
        int bits = 1;
        while (bits < 32 && ((int64_t)1 << bits) < G + 1) ++bits;
        bool in1b = false;
        BR(radix_sort_pairs(kb, va, kc, vb, kb, va, n_dev, L, bits, false, n_dev + 1, sw, &in1b, st));
        const uint32_t* gk = in1b ? kc : kb;
        const uint32_t* gv = in1b ? vb : va;
        assign_kernel<<<grid, 256, 0, st>>>(n_active, gk, gv, d_start, d_cnt, d_next, seg, leaf_of_node);
        BR(cudaMemcpyAsync(perm, gv, 4 * (size_t)L, cudaMemcpyDeviceToDevice, st));
        BR(cudaGetLastError());
        BR(cudaStreamSynchronize(st));  // the host arrays of this level are reused by the next one
    }
    leaf_nodes_kernel<<<grid, 256, 0, st>>>(N, out.child_count, leaf_of_node, mean, scale, rot, opacity, sh, lbox, work,
                                            ebox);
    BR(cudaGetLastError());
    for (int d = n_levels - 1; d >= 0; --d) {
        const int64_t G = (int64_t)lvl_nodes[d].size();
        if (G == 0) continue;
        BR(cudaMemcpyAsync(d_nodes, lvl_nodes[d].data(), 4 * G, cudaMemcpyHostToDevice, st));
        merge_kernel<<<(unsigned)std::min<int64_t>((G + 127) / 128, grid), 128, 0, st>>>(G, d_nodes, out.child_start, work);
        BR(cudaGetLastError());
        BR(cudaStreamSynchronize(st));
    }
    for (int d = 0; d < n_levels; ++d) {
        const int64_t G = (int64_t)lvl_nodes[d].size();
        if (G == 0) continue;
        BR(cudaMemcpyAsync(d_nodes, lvl_nodes[d].data(), 4 * G, cudaMemcpyHostToDevice, st));
        orient_kernel<<<(unsigned)std::min<int64_t>((G + 127) / 128, grid), 128, 0, st>>>(G, d_nodes, out.child_start,
                                                                                      out.child_count, work,
                                                                                      ex.orient_leaves ? 1 : 0);
        BR(cudaGetLastError());
        BR(cudaStreamSynchronize(st));
    }
    output_kernel<<<grid, 256, 0, st>>>(N, work, ebox, out.mean, out.scale, out.rot, out.opacity, out.sh, out.box_min,
                                        out.box_max);
    if (ex.leaf_node) leaf_node_kernel<<<grid, 256, 0, st>>>(N, out.child_count, leaf_of_node, ex.leaf_node);
    BR(cudaGetLastError());
    BR(cudaStreamSynchronize(st));
    return cudaSuccess;
}

namespace {

// local node j >= 1 of a chunk's hierarchy -> global node base + j - 1; the root's children keep
// parent -1 until the top tree is known (patched by chunk_root_kernel)
__global__ void chunk_copy_kernel(int64_t Nc, BuildOut src, BuildOut dst, int64_t base) {
    for (int64_t j = 1 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < Nc; j += (int64_t)gridDim.x * blockDim.x) {
        const int64_t g = base + j - 1;
        for (int k = 0; k < 3; ++k) {
            dst.mean[3 * g + k] = src.mean[3 * j + k];
            dst.scale[3 * g + k] = src.scale[3 * j + k];
            dst.box_min[3 * g + k] = src.box_min[3 * j + k];
            dst.box_max[3 * g + k] = src.box_max[3 * j + k];
        }
        for (int k = 0; k < 4; ++k) dst.rot[4 * g + k] = src.rot[4 * j + k];
        dst.opacity[g] = src.opacity[j];
        for (int c = 0; c < NSH; ++c) dst.sh[NSH * g + c] = src.sh[NSH * j + c];
        const int32_t p = src.parent[j], cs = src.child_start[j];
        dst.parent[g] = p == 0 ? -1 : (int32_t)(base + p - 1);
        dst.child_start[g] = cs >= 0 ? (int32_t)(base + cs - 1) : -1;
        dst.child_count[g] = src.child_count[j];
    }
}

// the chunk root as a leaf of the top tree: its attributes and leaf-union box
__global__ void chunk_root_out_kernel(BuildOut src, int64_t c, float* mean, float* scale, float* rot, float* opacity,
                                      float* sh, float* box) {
    const int k = threadIdx.x;
    if (k < 3) {
        mean[3 * c + k] = src.mean[k];
        scale[3 * c + k] = src.scale[k];
        box[6 * c + k] = src.box_min[k];
        box[6 * c + 3 + k] = src.box_max[k];
    }
    if (k < 4) rot[4 * c + k] = src.rot[k];
    if (k == 0) opacity[c] = src.opacity[0];
    if (k < NSH) sh[NSH * c + k] = src.sh[k];
}

// link every chunk's root (a leaf of the top tree) with the chunk's first nodes
__global__ void chunk_root_kernel(int K, const int64_t* __restrict__ base, const int32_t* __restrict__ root_children,
                                  const int32_t* __restrict__ top_node, BuildOut dst) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < K; c += gridDim.x * blockDim.x) {
        const int32_t v = top_node[c], nc = root_children[c];
        if (nc == 0) continue;
        dst.child_start[v] = (int32_t)base[c];
        dst.child_count[v] = nc;
        for (int i = 0; i < nc; ++i) dst.parent[base[c] + i] = v;
    }
}

}  // namespace

cudaError_t build_hierarchy_chunked(int K, const int64_t* off, const float* mean, const float* scale, const float* rot,
                                    const float* opacity, const float* sh, const BuildOut& out, const SortWork& sw,
                                    int num_sms, cudaStream_t st) {
    int64_t Lmax = 0;
    for (int c = 0; c < K; ++c) Lmax = std::max<int64_t>(Lmax, off[c + 1] - off[c]);
    const int64_t Nmax = 2 * Lmax - 1;
    DevMem mem;
    BuildOut scr;
    BR(mem.alloc(&scr.mean, 3 * (size_t)Nmax));
    BR(mem.alloc(&scr.scale, 3 * (size_t)Nmax));
    BR(mem.alloc(&scr.rot, 4 * (size_t)Nmax));
    BR(mem.alloc(&scr.opacity, (size_t)Nmax));
    BR(mem.alloc(&scr.sh, (size_t)NSH * Nmax));
    BR(mem.alloc(&scr.box_min, 3 * (size_t)Nmax));
    BR(mem.alloc(&scr.box_max, 3 * (size_t)Nmax));
    BR(mem.alloc(&scr.parent, (size_t)Nmax));
    BR(mem.alloc(&scr.child_start, (size_t)Nmax));
    BR(mem.alloc(&scr.child_count, (size_t)Nmax));
    float *tm, *ts, *tr, *to, *tsh, *tb;
    int32_t *top_node, *root_children;
    int64_t* d_base;
    BR(mem.alloc(&tm, 3 * (size_t)K));
    BR(mem.alloc(&ts, 3 * (size_t)K));
    BR(mem.alloc(&tr, 4 * (size_t)K));
    BR(mem.alloc(&to, (size_t)K));
    BR(mem.alloc(&tsh, (size_t)NSH * K));
    BR(mem.alloc(&tb, 6 * (size_t)K));
    BR(mem.alloc(&top_node, (size_t)K));
    BR(mem.alloc(&root_children, (size_t)K));
    BR(mem.alloc(&d_base, (size_t)K));
    const int64_t Ntop = 2 * (int64_t)K - 1;
    std::vector<int64_t> base(K);
    std::vector<int32_t> rc(K);
    int64_t next = Ntop;
    const int grid = num_sms * 8;
    for (int c = 0; c < K; ++c) {
        const int64_t Lc = off[c + 1] - off[c];
        const int64_t o = off[c];
        BR(build_hierarchy(Lc, mean + 3 * o, scale + 3 * o, rot + 4 * o, opacity + o, sh + (int64_t)NSH * o, scr, sw,
                           num_sms, st));
        chunk_root_out_kernel<<<1, 64, 0, st>>>(scr, c, tm, ts, tr, to, tsh, tb);
        base[c] = next;
        rc[c] = Lc >= 2 ? 2 : 0;
        const int64_t Nc = 2 * Lc - 1;
        if (Nc > 1) {
            BuildOut dst = out;
            chunk_copy_kernel<<<(unsigned)std::min<int64_t>((Nc + 255) / 256, grid), 256, 0, st>>>(Nc, scr, dst, base[c]);
        }
        next += Nc - 1;
        BR(cudaGetLastError());
    }
    // the top tree over the chunk roots: leaf boxes are the chunks' leaf-union boxes, and the chunk
    // roots keep their own frames (no orientation matching at the chunk boundary)
    BuildExtra ex;
    ex.leaf_box = tb;
    ex.orient_leaves = false;
    ex.leaf_node = top_node;
    BR(build_hierarchy(K, tm, ts, tr, to, tsh, out, sw, num_sms, st, ex));
    BR(cudaMemcpyAsync(d_base, base.data(), sizeof(int64_t) * K, cudaMemcpyHostToDevice, st));
    BR(cudaMemcpyAsync(root_children, rc.data(), sizeof(int32_t) * K, cudaMemcpyHostToDevice, st));
    chunk_root_kernel<<<(K + 255) / 256, 256, 0, st>>>(K, d_base, root_children, top_node, out);
    BR(cudaGetLastError());
    BR(cudaStreamSynchronize(st));
    return cudaSuccess;
}

#undef BR

}  // namespace h3dgs
