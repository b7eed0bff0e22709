// TEST INFRASTRUCTURE ONLY -- the CPU oracle for the hierarchical 3D Gaussian render path.
//
// A plain, slow restatement of "A Hierarchical 3D Gaussian Representation for Real-Time
// Rendering of Very Large Datasets" (Kerbl et al. 2024): hierarchy merge (Sec. 4.1, Eq. merge),
// BVH build and orientation matching (Sec. 4.1-4.2), granularity / cut / interpolation weights
// (Sec. 4.2, Eq. t_interp), attribute interpolation and transition opacity (Sec. 4.2,
// Eq. alphap and its K-child form in Sec. 5.2), EWA-filtered splatting (Sec. 3.1 Eq. alpha,
// Sec. 5.1), front-to-back blending, and the analytic adjoint used by hierarchy optimisation
// (Sec. 5.1, Sec. 7.1, Sec. 7.3).  Only the tests, the smoke check and the benchmark's CPU-baseline leg
// call it; the product library never links or loads it, and the two share no code.
//
// Two tracks are computed side by side:
//  * the VALUE track, in fp64, produces everything continuous (colours, opacities, splat
//    geometry used for blending, images, gradients);
//  * the DECISION track, in fp32 with a fixed evaluation order (no contraction; fma only where
//    written as fmaf), takes every decision that turns floating point into an integer or a set:
//    cut membership, the interpolation weight t (it is a function of the cut test's
//    granularities), tile rectangles, depth keys, culling, and the per-pixel alpha-floor and
//    transmittance-stop tests.  Transcendentals in that track (exp2, pow) are evaluated in double
//    and rounded; a decision within a few ulps of its threshold is reported as ambiguous.
//
// Build: g++ -O2 -fopenmp -ffp-contract=off -fPIC -shared  (no -ffast-math: IEEE semantics).

#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>
#include <algorithm>
#include <numeric>
#include <array>

#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

constexpr int NSH = 48;          // 16 SH basis functions x 3 colour channels, layout [k*3 + ch]
constexpr int NATTR = 59;        // mean 3, scale 3, rot 4, opacity 1, sh 48
constexpr int NVAL = 13;         // value-track splat row: u v A B C on op t K r g b z
constexpr double PI = 3.14159265358979323846;

// ------------------------------------------------------------------------------------------
// Plain data structures (the oracle's own; nothing is shared with the CUDA library)
// ------------------------------------------------------------------------------------------

}  // namespace

extern "C" {

struct OrCamera {
    float R[9];      // world -> camera rotation, row-major
    float T[3];      // world -> camera translation: x_c = R x_w + T
    float fx, fy, cx, cy;
    int32_t width, height;
    float znear;
    float tau;       // target granularity in pixels
};

struct OrHier32 {    // fp32 node arrays as stored in the hierarchy file
    int64_t n;
    const float *mean, *scale, *rot, *opacity, *sh;   // [N,3] [N,3] [N,4] (w,x,y,z) [N] [N,48]
    const float *box_min, *box_max;                   // [N,3]
    const int32_t *parent, *child_start, *child_count;
};

struct OrHier64 {    // the same attributes in double (value track; perturbed by FD checks)
    const double *mean, *scale, *rot, *opacity, *sh;
};

struct OrOpts {
    int32_t tile_w, tile_h;
    float lowpass;          // screen-space low-pass variance added to the 2D covariance (px^2)
    int32_t aa_compensate;  // multiply opacities by sqrt(det S' / det (S' + lowpass I))
    int32_t interpolate;    // 0: t = 0 everywhere (interpolation off)
    float alpha_clamp;      // 0.99
    float alpha_floor;      // 1/255
    float t_min;            // transmittance stop threshold, 1e-4
    float bg[3];
};

}  // extern "C"

namespace {

// ------------------------------------------------------------------------------------------
// Small fp64 linear algebra
// ------------------------------------------------------------------------------------------

struct M3 { double a[3][3]; };

M3 quat_to_mat(const double q_in[4]) {
    // q = (w, x, y, z); normalised first.  Standard rotation matrix of a unit quaternion.
    double n = std::sqrt(q_in[0] * q_in[0] + q_in[1] * q_in[1] + q_in[2] * q_in[2] + q_in[3] * q_in[3]);
    double w = q_in[0] / n, x = q_in[1] / n, y = q_in[2] / n, z = q_in[3] / n;
    M3 r;
    r.a[0][0] = 1 - 2 * (y * y + z * z); r.a[0][1] = 2 * (x * y - w * z);     r.a[0][2] = 2 * (x * z + w * y);
    r.a[1][0] = 2 * (x * y + w * z);     r.a[1][1] = 1 - 2 * (x * x + z * z); r.a[1][2] = 2 * (y * z - w * x);
    r.a[2][0] = 2 * (x * z - w * y);     r.a[2][1] = 2 * (y * z + w * x);     r.a[2][2] = 1 - 2 * (x * x + y * y);
    return r;
}

void mat_to_quat(const M3& m, double q[4]) {
    // Shepperd's method: pick the largest of (w, x, y, z) to divide by.
    const auto& R = m.a;
    double tr = R[0][0] + R[1][1] + R[2][2];
    if (tr > 0) {
        double S = std::sqrt(tr + 1.0) * 2;
        q[0] = 0.25 * S; q[1] = (R[2][1] - R[1][2]) / S; q[2] = (R[0][2] - R[2][0]) / S; q[3] = (R[1][0] - R[0][1]) / S;
    } else if (R[0][0] > R[1][1] && R[0][0] > R[2][2]) {
        double S = std::sqrt(1.0 + R[0][0] - R[1][1] - R[2][2]) * 2;
        q[0] = (R[2][1] - R[1][2]) / S; q[1] = 0.25 * S; q[2] = (R[0][1] + R[1][0]) / S; q[3] = (R[0][2] + R[2][0]) / S;
    } else if (R[1][1] > R[2][2]) {
        double S = std::sqrt(1.0 + R[1][1] - R[0][0] - R[2][2]) * 2;
        q[0] = (R[0][2] - R[2][0]) / S; q[1] = (R[0][1] + R[1][0]) / S; q[2] = 0.25 * S; q[3] = (R[1][2] + R[2][1]) / S;
    } else {
        double S = std::sqrt(1.0 + R[2][2] - R[0][0] - R[1][1]) * 2;
        q[0] = (R[1][0] - R[0][1]) / S; q[1] = (R[0][2] + R[2][0]) / S; q[2] = (R[1][2] + R[2][1]) / S; q[3] = 0.25 * S;
    }
    double n = std::sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    for (int i = 0; i < 4; ++i) q[i] /= n;
}

// Covariance Sigma = R diag(s^2) R^T of a Gaussian given scale and quaternion.
M3 covariance(const double s[3], const double q[4]) {
    M3 R = quat_to_mat(q), C;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double acc = 0;
            for (int k = 0; k < 3; ++k) acc += R.a[i][k] * s[k] * s[k] * R.a[j][k];
            C.a[i][j] = acc;
        }
    return C;
}

// Cyclic Jacobi eigen-decomposition of a symmetric 3x3 matrix (textbook algorithm).
// Returns eigenvalues in lam and eigenvectors as the COLUMNS of V.
void jacobi_eigen(M3 A, double lam[3], M3& V) {
    for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) V.a[i][j] = (i == j);
    for (int sweep = 0; sweep < 64; ++sweep) {
        double off = A.a[0][1] * A.a[0][1] + A.a[0][2] * A.a[0][2] + A.a[1][2] * A.a[1][2];
        double diag = A.a[0][0] * A.a[0][0] + A.a[1][1] * A.a[1][1] + A.a[2][2] * A.a[2][2];
        if (off <= 1e-40 * diag || off == 0.0) break;
        for (int p = 0; p < 2; ++p)
            for (int q = p + 1; q < 3; ++q) {
                double apq = A.a[p][q];
                if (apq == 0.0) continue;
                double theta = (A.a[q][q] - A.a[p][p]) / (2 * apq);
                double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1));
                double c = 1 / std::sqrt(t * t + 1), s = t * c;
                // A <- J^T A J with J the rotation in the (p, q) plane
                for (int k = 0; k < 3; ++k) {
                    double akp = A.a[k][p], akq = A.a[k][q];
                    A.a[k][p] = c * akp - s * akq;
                    A.a[k][q] = s * akp + c * akq;
                }
                for (int k = 0; k < 3; ++k) {
                    double apk = A.a[p][k], aqk = A.a[q][k];
                    A.a[p][k] = c * apk - s * aqk;
                    A.a[q][k] = s * apk + c * aqk;
                }
                for (int k = 0; k < 3; ++k) {
                    double vkp = V.a[k][p], vkq = V.a[k][q];
                    V.a[k][p] = c * vkp - s * vkq;
                    V.a[k][q] = s * vkp + c * vkq;
                }
            }
    }
    for (int i = 0; i < 3; ++i) lam[i] = A.a[i][i];
}

// Surface area of an ellipsoid with semi-axes a, b, c (Knud Thomsen's approximation,
// p = 1.6075, max relative error ~1.06%).  Stands in for sqrt|Sigma'| in the merge weights.
double ellipsoid_area(const double s[3]) {
    const double p = 1.6075;
    double ap = std::pow(s[0], p), bp = std::pow(s[1], p), cp = std::pow(s[2], p);
    return 4 * PI * std::pow((ap * bp + ap * cp + bp * cp) / 3.0, 1.0 / p);
}

struct G64 { double mu[3], s[3], q[4], o, sh[NSH]; };

// Sec. 4.1, Eq. merge with weights w'_i = o_i S_i (S_i the ellipsoid surface), normalised;
// SH merged with the same weights; the parent's opacity becomes the falloff sum(w'_i) / S_p.
G64 merge(const std::vector<const G64*>& ch) {
    const size_t K = ch.size();
    std::vector<double> wp(K);
    double W = 0;
    for (size_t i = 0; i < K; ++i) { wp[i] = ch[i]->o * ellipsoid_area(ch[i]->s); W += wp[i]; }
    std::vector<double> w(K);
    for (size_t i = 0; i < K; ++i) w[i] = (W > 0) ? wp[i] / W : 1.0 / K;
    G64 p{};
    for (size_t i = 0; i < K; ++i)
        for (int d = 0; d < 3; ++d) p.mu[d] += w[i] * ch[i]->mu[d];
    M3 S{};
    for (size_t i = 0; i < K; ++i) {
        M3 Ci = covariance(ch[i]->s, ch[i]->q);
        double dm[3] = {ch[i]->mu[0] - p.mu[0], ch[i]->mu[1] - p.mu[1], ch[i]->mu[2] - p.mu[2]};
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) S.a[a][b] += w[i] * (Ci.a[a][b] + dm[a] * dm[b]);
    }
    for (size_t i = 0; i < K; ++i)
        for (int c = 0; c < NSH; ++c) p.sh[c] += w[i] * ch[i]->sh[c];
    double lam[3];
    M3 V;
    jacobi_eigen(S, lam, V);
    // order the eigen-axes by decreasing eigenvalue, then make the frame right-handed
    int ord[3] = {0, 1, 2};
    std::sort(ord, ord + 3, [&](int x, int y) { return lam[x] > lam[y]; });
    M3 Rm;
    for (int j = 0; j < 3; ++j) {
        p.s[j] = std::sqrt(std::max(lam[ord[j]], 0.0));
        for (int i = 0; i < 3; ++i) Rm.a[i][j] = V.a[i][ord[j]];
    }
    double det = Rm.a[0][0] * (Rm.a[1][1] * Rm.a[2][2] - Rm.a[1][2] * Rm.a[2][1])
               - Rm.a[0][1] * (Rm.a[1][0] * Rm.a[2][2] - Rm.a[1][2] * Rm.a[2][0])
               + Rm.a[0][2] * (Rm.a[1][0] * Rm.a[2][1] - Rm.a[1][1] * Rm.a[2][0]);
    if (det < 0) for (int i = 0; i < 3; ++i) Rm.a[i][2] = -Rm.a[i][2];
    mat_to_quat(Rm, p.q);
    double Sp = ellipsoid_area(p.s);
    p.o = (Sp > 0) ? W / Sp : 0.0;
    return p;
}

// The 24 proper signed axis permutations, enumerated in a fixed order: permutations of
// (0,1,2) in lexicographic order, sign patterns in binary order (+ before -), det = +1 only.
struct SignedPerm { int perm[3]; double sign[3]; };
std::vector<SignedPerm> proper_signed_perms() {
    std::vector<SignedPerm> out;
    int p[3] = {0, 1, 2};
    do {
        int inv = 0;
        for (int i = 0; i < 3; ++i) for (int j = i + 1; j < 3; ++j) inv += p[i] > p[j];
        double psign = (inv % 2) ? -1.0 : 1.0;
        for (int bits = 0; bits < 8; ++bits) {
            SignedPerm sp;
            for (int i = 0; i < 3; ++i) { sp.perm[i] = p[i]; sp.sign[i] = (bits >> (2 - i)) & 1 ? -1.0 : 1.0; }
            if (psign * sp.sign[0] * sp.sign[1] * sp.sign[2] > 0) out.push_back(sp);
        }
    } while (std::next_permutation(p, p + 3));
    return out;
}

// Sec. 4.2, orientation matching: reinterpret the child's axes (a signed permutation of the
// columns of its rotation, scales permuted alike) to minimise the rotation relative to the
// parent, by exhaustive search; the quaternion sign is then aligned with the parent's.
void match_orientation(const G64& parent, G64& child) {
    static const std::vector<SignedPerm> perms = proper_signed_perms();
    M3 Rp = quat_to_mat(parent.q), Rc = quat_to_mat(child.q);
    int best = 0;
    double best_tr = -1e300;
    for (size_t k = 0; k < perms.size(); ++k) {
        double tr = 0;
        for (int j = 0; j < 3; ++j)
            for (int i = 0; i < 3; ++i) tr += Rp.a[i][j] * perms[k].sign[j] * Rc.a[i][perms[k].perm[j]];
        if (tr > best_tr) { best_tr = tr; best = (int)k; }
    }
    const SignedPerm& P = perms[best];
    M3 Rn;
    double sn[3];
    for (int j = 0; j < 3; ++j) {
        sn[j] = child.s[P.perm[j]];
        for (int i = 0; i < 3; ++i) Rn.a[i][j] = P.sign[j] * Rc.a[i][P.perm[j]];
    }
    mat_to_quat(Rn, child.q);
    for (int j = 0; j < 3; ++j) child.s[j] = sn[j];
    double dot = 0;
    for (int i = 0; i < 4; ++i) dot += child.q[i] * parent.q[i];
    if (dot < 0) for (int i = 0; i < 4; ++i) child.q[i] = -child.q[i];
}

}  // namespace

// ==========================================================================================
// Hierarchy construction (Sec. 4.1)
// ==========================================================================================

extern "C" {

// Returns the angle (radians) between the rotations of two quaternions, used by tests to
// check that orientation matching picks the smallest of the 24 alternatives.
double or_rotation_angle(const double* qa, const double* qb) {
    M3 A = quat_to_mat(qa), B = quat_to_mat(qb);
    double tr = 0;
    for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) tr += A.a[i][j] * B.a[i][j];
    double c = std::max(-1.0, std::min(1.0, (tr - 1) / 2));
    return std::acos(c);
}

// Merge K Gaussians (double attributes, rows of 59 = mean 3, scale 3, rot 4, opacity 1, sh 48)
// into one parent row (same layout).  Exposed for the closed-form tests.
void or_merge(int32_t K, const double* rows, double* out) {
    std::vector<G64> g(K);
    std::vector<const G64*> ptr(K);
    for (int i = 0; i < K; ++i) {
        const double* r = rows + (size_t)i * NATTR;
        for (int d = 0; d < 3; ++d) { g[i].mu[d] = r[d]; g[i].s[d] = r[3 + d]; }
        for (int d = 0; d < 4; ++d) g[i].q[d] = r[6 + d];
        g[i].o = r[10];
        for (int c = 0; c < NSH; ++c) g[i].sh[c] = r[11 + c];
        ptr[i] = &g[i];
    }
    G64 p = merge(ptr);
    for (int d = 0; d < 3; ++d) { out[d] = p.mu[d]; out[3 + d] = p.s[d]; }
    for (int d = 0; d < 4; ++d) out[6 + d] = p.q[d];
    out[10] = p.o;
    for (int c = 0; c < NSH; ++c) out[11 + c] = p.sh[c];
}

void or_match_orientation(const double* parent_row, double* child_row) {
    G64 p{}, c{};
    for (int d = 0; d < 3; ++d) { p.mu[d] = parent_row[d]; p.s[d] = parent_row[3 + d]; c.mu[d] = child_row[d]; c.s[d] = child_row[3 + d]; }
    for (int d = 0; d < 4; ++d) { p.q[d] = parent_row[6 + d]; c.q[d] = child_row[6 + d]; }
    match_orientation(p, c);
    for (int d = 0; d < 3; ++d) child_row[3 + d] = c.s[d];
    for (int d = 0; d < 4; ++d) child_row[6 + d] = c.q[d];
}

// Build the hierarchy over n_items leaf Gaussians.
//
// BVH (Sec. 4.1): boxes are the 3-sigma AABBs of the leaves; a group's box is the union of its
// members' boxes; the group is split at the median of the members' means projected on the
// longest box axis (ties to the lower axis index; members ordered by (projected mean, item
// index); the left child takes the first floor(n/2)).  Nodes are numbered breadth-first: root 0,
// children contiguous, parent < child.  Attributes are merged bottom-up from the direct
// children; orientation matching runs top-down from the root.
//
// Outputs are fp32 arrays sized for n_out nodes.  Returns the node count, or -1 on bad input.
int64_t or_build_tree(int64_t n_items,
                      const float* mean, const float* scale, const float* rot, const float* opacity,
                      const float* sh,
                      float* o_mean, float* o_scale, float* o_rot, float* o_opacity, float* o_sh,
                      float* o_box_min, float* o_box_max, int32_t* o_parent, int32_t* o_child_start,
                      int32_t* o_child_count) {
    if (n_items <= 0) return -1;
    const int64_t L = n_items;
    // leaf 3-sigma boxes, computed in double and rounded to fp32 once
    std::vector<float> lbmin(3 * L), lbmax(3 * L);
    std::vector<G64> leaf(L);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < L; ++i) {
        G64& g = leaf[i];
        for (int d = 0; d < 3; ++d) { g.mu[d] = mean[3 * i + d]; g.s[d] = scale[3 * i + d]; }
        for (int d = 0; d < 4; ++d) g.q[d] = rot[4 * i + d];
        g.o = opacity[i];
        for (int c = 0; c < NSH; ++c) g.sh[c] = sh[(size_t)NSH * i + c];
        M3 R = quat_to_mat(g.q);
        for (int j = 0; j < 3; ++j) {
            double v = 0;
            for (int k = 0; k < 3; ++k) v += (R.a[j][k] * g.s[k]) * (R.a[j][k] * g.s[k]);
            double h = 3.0 * std::sqrt(v);
            lbmin[3 * i + j] = (float)(g.mu[j] - h);
            lbmax[3 * i + j] = (float)(g.mu[j] + h);
        }
    }
    // breadth-first median-split BVH over a permutation of the items
    std::vector<int64_t> perm(L);
    std::iota(perm.begin(), perm.end(), 0);
    struct Node { int64_t lo, hi; int64_t first_child; int32_t nchild; int64_t parent; };
    std::vector<Node> nodes;
    nodes.reserve(2 * L);
    nodes.push_back({0, L, -1, 0, -1});
    for (size_t cur = 0; cur < nodes.size(); ++cur) {
        int64_t lo = nodes[cur].lo, hi = nodes[cur].hi, n = hi - lo;
        if (n < 2) continue;
        float bmin[3] = {INFINITY, INFINITY, INFINITY}, bmax[3] = {-INFINITY, -INFINITY, -INFINITY};
        for (int64_t k = lo; k < hi; ++k)
            for (int d = 0; d < 3; ++d) {
                bmin[d] = std::min(bmin[d], lbmin[3 * perm[k] + d]);
                bmax[d] = std::max(bmax[d], lbmax[3 * perm[k] + d]);
            }
        int axis = 0;
        double ext = (double)bmax[0] - (double)bmin[0];
        for (int d = 1; d < 3; ++d) {
            double e = (double)bmax[d] - (double)bmin[d];
            if (e > ext) { ext = e; axis = d; }
        }
        std::sort(perm.begin() + lo, perm.begin() + hi, [&](int64_t a, int64_t b) {
            float ma = mean[3 * a + axis], mb = mean[3 * b + axis];
            return ma < mb || (ma == mb && a < b);
        });
        int64_t mid = lo + n / 2;
        nodes[cur].first_child = (int64_t)nodes.size();
        nodes[cur].nchild = 2;
        nodes.push_back({lo, mid, -1, 0, (int64_t)cur});
        nodes.push_back({mid, hi, -1, 0, (int64_t)cur});
    }
    const int64_t N = (int64_t)nodes.size();
    std::vector<G64> g(N);
    std::vector<float> bmin(3 * N), bmax(3 * N);
    // bottom-up: leaves take their Gaussian and box; interior nodes merge their children
    for (int64_t v = N - 1; v >= 0; --v) {
        const Node& nd = nodes[v];
        if (nd.nchild == 0) {
            int64_t li = perm[nd.lo];
            g[v] = leaf[li];
            for (int d = 0; d < 3; ++d) { bmin[3 * v + d] = lbmin[3 * li + d]; bmax[3 * v + d] = lbmax[3 * li + d]; }
        } else {
            std::vector<const G64*> ch;
            for (int c = 0; c < nd.nchild; ++c) ch.push_back(&g[nd.first_child + c]);
            g[v] = merge(ch);
            for (int d = 0; d < 3; ++d) {
                float lo = INFINITY, hi = -INFINITY;
                for (int c = 0; c < nd.nchild; ++c) {
                    lo = std::min(lo, bmin[3 * (nd.first_child + c) + d]);
                    hi = std::max(hi, bmax[3 * (nd.first_child + c) + d]);
                }
                bmin[3 * v + d] = lo; bmax[3 * v + d] = hi;
            }
        }
    }
    // top-down orientation matching (the root keeps its eigen-frame)
    for (int64_t v = 0; v < N; ++v)
        for (int c = 0; c < nodes[v].nchild; ++c) match_orientation(g[v], g[nodes[v].first_child + c]);
    for (int64_t v = 0; v < N; ++v) {
        for (int d = 0; d < 3; ++d) {
            o_mean[3 * v + d] = (float)g[v].mu[d];
            o_scale[3 * v + d] = (float)g[v].s[d];
            o_box_min[3 * v + d] = bmin[3 * v + d];
            o_box_max[3 * v + d] = bmax[3 * v + d];
        }
        for (int d = 0; d < 4; ++d) o_rot[4 * v + d] = (float)g[v].q[d];
        o_opacity[v] = (float)g[v].o;
        for (int c = 0; c < NSH; ++c) o_sh[(size_t)NSH * v + c] = (float)g[v].sh[c];
        o_parent[v] = (int32_t)nodes[v].parent;
        o_child_start[v] = nodes[v].nchild ? (int32_t)nodes[v].first_child : -1;
        o_child_count[v] = nodes[v].nchild;
    }
    return N;
}

}  // extern "C"

// ==========================================================================================
// Decision track: granularity and cut (Sec. 4.2), fp32 in a fixed order
// ==========================================================================================

namespace {

struct CamF { float c[3]; float f; };

CamF camera_center_f(const OrCamera& cam) {
    // c = -R^T T, each component as fmaf(R2j, T2, fmaf(R1j, T1, R0j * T0)), negated
    CamF out;
    for (int j = 0; j < 3; ++j) {
        float acc = cam.R[0 * 3 + j] * cam.T[0];
        acc = fmaf(cam.R[1 * 3 + j], cam.T[1], acc);
        acc = fmaf(cam.R[2 * 3 + j], cam.T[2], acc);
        out.c[j] = -acc;
    }
    out.f = std::max(cam.fx, cam.fy);
    return out;
}

// Granularity: projected size of the node's leaf-union box (largest box dimension), measured at
// the box's closest point to the camera centre.  +inf when the camera is inside the box.
float granularity_f(const CamF& cf, const float* lo, const float* hi) {
    float d[3];
    for (int k = 0; k < 3; ++k) {
        float a = lo[k] - cf.c[k];
        float b = cf.c[k] - hi[k];
        d[k] = std::max(std::max(a, b), 0.0f);
    }
    float dist2 = d[0] * d[0];
    dist2 = fmaf(d[1], d[1], dist2);
    dist2 = fmaf(d[2], d[2], dist2);
    float size = std::max(std::max(hi[0] - lo[0], hi[1] - lo[1]), hi[2] - lo[2]);
    if (dist2 == 0.0f) return INFINITY;
    return (cf.f * size) / std::sqrt(dist2);
}

// Interpolation weight t (the PARENT's weight): (tau - eps_n) / (eps_p - eps_n) when the node
// passed the test with a finite parent granularity; 0 otherwise (root, forced leaf, eps_p = inf).
float weight_f(float tau, float en, float ep) {
    if (!(en < tau) || !(ep >= tau) || std::isinf(ep)) return 0.0f;
    float t = (tau - en) / (ep - en);
    return std::min(std::max(t, 0.0f), 1.0f);
}

}  // namespace

extern "C" {

void or_granularity(const OrCamera* cam, const OrHier32* h, float* eps) {
    CamF cf = camera_center_f(*cam);
#pragma omp parallel for schedule(static)
    for (int64_t v = 0; v < h->n; ++v) eps[v] = granularity_f(cf, h->box_min + 3 * v, h->box_max + 3 * v);
}

// Cut (Sec. 4.2): node n is in the cut iff (eps(n) < tau or n is a leaf) and (n is the root or
// eps(parent) >= tau).  Ids are written in ascending order with the parent weight t.
// Returns the cut size (only the first `cap` entries are written).
int64_t or_select_cut(const OrCamera* cam, const OrHier32* h, int32_t interpolate, int32_t* ids,
                      float* t, int64_t cap) {
    CamF cf = camera_center_f(*cam);
    const float tau = cam->tau;
    int64_t m = 0;
    for (int64_t v = 0; v < h->n; ++v) {
        float en = granularity_f(cf, h->box_min + 3 * v, h->box_max + 3 * v);
        bool leaf = h->child_count[v] == 0;
        bool self_ok = (en < tau) || leaf;
        int32_t p = h->parent[v];
        float ep = INFINITY;
        bool parent_ok = true;
        if (p >= 0) {
            ep = granularity_f(cf, h->box_min + 3 * (int64_t)p, h->box_max + 3 * (int64_t)p);
            parent_ok = ep >= tau;
        }
        if (self_ok && parent_ok) {
            if (m < cap) {
                ids[m] = (int32_t)v;
                if (t) t[m] = (interpolate && p >= 0) ? weight_f(tau, en, ep) : 0.0f;
            }
            ++m;
        }
    }
    return m;
}

// The same cut found by a recursive descent from the root (expand while eps >= tau and the node
// has children).  Used by the tests to cross-check the constant-time-per-node rule.
int64_t or_select_cut_descent(const OrCamera* cam, const OrHier32* h, int32_t* ids, int64_t cap) {
    CamF cf = camera_center_f(*cam);
    std::vector<int64_t> stack = {0}, out;
    while (!stack.empty()) {
        int64_t v = stack.back();
        stack.pop_back();
        float e = granularity_f(cf, h->box_min + 3 * v, h->box_max + 3 * v);
        if (e < cam->tau || h->child_count[v] == 0) out.push_back(v);
        else for (int c = 0; c < h->child_count[v]; ++c) stack.push_back((int64_t)h->child_start[v] + c);
    }
    std::sort(out.begin(), out.end());
    for (size_t i = 0; i < out.size() && (int64_t)i < cap; ++i) ids[i] = (int32_t)out[i];
    return (int64_t)out.size();
}

// Hierarchy compaction (Sec. 5.2), step by step as the paper describes it.
//   * The leaves start out marked as relevant.
//   * For tau = tau_min, 2 tau_min, 4 tau_min, ... (doubled in fp32) while tau <= tau_max:
//       U = the union over the training views of their cuts at tau;
//       B = the bottom-most members of U (no member of U strictly below them);
//       every node strictly below a node of B that is not yet marked is removed;
//       the nodes of B are marked.
//   * A kept node's new parent is its closest kept ancestor (a node can now have K > 2 children).
//   * Kept nodes are renumbered breadth-first from the root; siblings keep their old relative order.
// Outputs are indexed by the new numbering; old_of_new[i] is the old index of new node i.
// Returns the number of kept nodes, or -1 for tau_min <= 0 or a non-finite tau_max.
int64_t or_compact(const OrCamera* cams, int32_t n_cams, const OrHier32* h, float tau_min, float tau_max,
                   int32_t* old_of_new, int32_t* new_parent, int32_t* new_child_start, int32_t* new_child_count) {
    if (!(tau_min > 0.0f) || !std::isfinite(tau_max)) return -1;
    const int64_t N = h->n;
    std::vector<char> marked(N), removed(N, 0), in_union(N), has_below(N), bottom(N), below(N);
    for (int64_t v = 0; v < N; ++v) marked[v] = h->child_count[v] == 0;
    std::vector<int32_t> ids(N);
    for (float tau = tau_min; tau <= tau_max; tau = tau * 2.0f) {
        std::fill(in_union.begin(), in_union.end(), 0);
        for (int32_t k = 0; k < n_cams; ++k) {
            OrCamera c = cams[k];
            c.tau = tau;
            const int64_t m = or_select_cut(&c, h, 0, ids.data(), nullptr, N);
            for (int64_t i = 0; i < m; ++i) in_union[ids[i]] = 1;
        }
        // children come after their parent, so one backward sweep sees every subtree before its root
        std::fill(has_below.begin(), has_below.end(), 0);
        for (int64_t v = N - 1; v > 0; --v)
            if (in_union[v] || has_below[v]) has_below[h->parent[v]] = 1;
        for (int64_t v = 0; v < N; ++v) bottom[v] = in_union[v] && !has_below[v];
        below[0] = 0;
        for (int64_t v = 1; v < N; ++v) {
            const int32_t p = h->parent[v];
            below[v] = bottom[p] || below[p];
        }
        for (int64_t v = 0; v < N; ++v)
            if (below[v] && !marked[v]) removed[v] = 1;
        for (int64_t v = 0; v < N; ++v)
            if (bottom[v]) marked[v] = 1;
    }
    std::vector<int32_t> up(N, -1);
    std::vector<std::vector<int32_t>> kids(N);
    for (int64_t v = 1; v < N; ++v) {
        if (removed[v]) continue;
        int32_t p = h->parent[v];
        while (removed[p]) p = h->parent[p];
        up[v] = p;
        kids[p].push_back((int32_t)v);
    }
    std::vector<int32_t> order = {0}, new_of_old(N, -1);
    new_of_old[0] = 0;
    for (size_t i = 0; i < order.size(); ++i)
        for (int32_t c : kids[order[i]]) {
            new_of_old[c] = (int32_t)order.size();
            order.push_back(c);
        }
    for (size_t i = 0; i < order.size(); ++i) {
        const int32_t o = order[i];
        old_of_new[i] = o;
        new_parent[i] = i == 0 ? -1 : new_of_old[up[o]];
        new_child_count[i] = (int32_t)kids[o].size();
        new_child_start[i] = kids[o].empty() ? -1 : new_of_old[kids[o][0]];
    }
    return (int64_t)order.size();
}

}  // extern "C"

// ==========================================================================================
// Interpolation (Sec. 4.2) and projection (Sec. 3.1, EWA low-pass of Sec. 5.1)
// ==========================================================================================

namespace {

// Interpolated attributes of one cut node.  Layout of the exported row (62 values):
//   mean 3 | scale 3 | rot 4 (normalised) | sh 48 | o_n | o_p | t | K
// o_p and K (the parent's opacity and child count) are 0 and 1 when t = 0 (they are unused).
constexpr int NINTERP = 62;

// fp32 track: a = fmaf(t, a_p, (1 - t) * a_n) for mean, scale, rot (then normalised), sh.
void interp_f(const OrHier32& h, int64_t n, float t, float out[NINTERP]) {
    int32_t p = h.parent[n];
    const float omt = 1.0f - t;
    auto lerp = [&](float an, float ap) { return fmaf(t, ap, omt * an); };
    bool use_p = (t != 0.0f) && p >= 0;
    for (int d = 0; d < 3; ++d) {
        out[d] = use_p ? lerp(h.mean[3 * n + d], h.mean[3 * (int64_t)p + d]) : h.mean[3 * n + d];
        out[3 + d] = use_p ? lerp(h.scale[3 * n + d], h.scale[3 * (int64_t)p + d]) : h.scale[3 * n + d];
    }
    float q[4];
    for (int d = 0; d < 4; ++d) q[d] = use_p ? lerp(h.rot[4 * n + d], h.rot[4 * (int64_t)p + d]) : h.rot[4 * n + d];
    float n2 = q[0] * q[0];
    n2 = fmaf(q[1], q[1], n2);
    n2 = fmaf(q[2], q[2], n2);
    n2 = fmaf(q[3], q[3], n2);
    if (n2 > 0.0f) {
        float nr = std::sqrt(n2);
        for (int d = 0; d < 4; ++d) out[6 + d] = q[d] / nr;
    } else {
        out[6] = 1.0f; out[7] = out[8] = out[9] = 0.0f;
    }
    for (int c = 0; c < NSH; ++c)
        out[10 + c] = use_p ? lerp(h.sh[(size_t)NSH * n + c], h.sh[(size_t)NSH * p + c]) : h.sh[(size_t)NSH * n + c];
    out[58] = h.opacity[n];
    out[59] = use_p ? h.opacity[p] : 0.0f;
    out[60] = t;
    out[61] = use_p ? (float)h.child_count[p] : 1.0f;
}

// fp64 track of the same interpolation (t is the fp32 weight, exactly representable).
void interp_d(const OrHier32& h, const OrHier64& hd, int64_t n, double t, double out[NINTERP]) {
    int32_t p = h.parent[n];
    bool use_p = (t != 0.0) && p >= 0;
    auto lerp = [&](double an, double ap) { return (1.0 - t) * an + t * ap; };
    for (int d = 0; d < 3; ++d) {
        out[d] = use_p ? lerp(hd.mean[3 * n + d], hd.mean[3 * (int64_t)p + d]) : hd.mean[3 * n + d];
        out[3 + d] = use_p ? lerp(hd.scale[3 * n + d], hd.scale[3 * (int64_t)p + d]) : hd.scale[3 * n + d];
    }
    double q[4];
    for (int d = 0; d < 4; ++d) q[d] = use_p ? lerp(hd.rot[4 * n + d], hd.rot[4 * (int64_t)p + d]) : hd.rot[4 * n + d];
    double nr = std::sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    if (nr > 0) for (int d = 0; d < 4; ++d) out[6 + d] = q[d] / nr;
    else { out[6] = 1; out[7] = out[8] = out[9] = 0; }
    for (int c = 0; c < NSH; ++c)
        out[10 + c] = use_p ? lerp(hd.sh[(size_t)NSH * n + c], hd.sh[(size_t)NSH * p + c]) : hd.sh[(size_t)NSH * n + c];
    out[58] = hd.opacity[n];
    out[59] = use_p ? hd.opacity[p] : 0.0;
    out[60] = t;
    out[61] = use_p ? (double)h.child_count[p] : 1.0;
}

// Real spherical harmonics up to degree 3 for a unit direction (x, y, z), orthonormal on the
// sphere, in the order l = 0..3, m = -l..l, with the Condon-Shortley phase.  Constants are the
// closed-form normalisations sqrt((2l+1)/(4 pi) (l-|m|)!/(l+|m|)!) (x sqrt 2 for m != 0).
void sh_basis(double x, double y, double z, double Y[16]) {
    const double c0 = 0.5 * std::sqrt(1.0 / PI);
    const double c1 = std::sqrt(3.0 / (4 * PI));
    const double c2a = std::sqrt(15.0 / (4 * PI)), c2b = std::sqrt(5.0 / (16 * PI)), c2c = std::sqrt(15.0 / (16 * PI));
    const double c3a = std::sqrt(35.0 / (32 * PI)), c3b = std::sqrt(105.0 / (4 * PI)), c3c = std::sqrt(21.0 / (32 * PI));
    const double c3d = std::sqrt(7.0 / (16 * PI)), c3e = std::sqrt(105.0 / (16 * PI));
    double xx = x * x, yy = y * y, zz = z * z;
    Y[0] = c0;
    Y[1] = -c1 * y; Y[2] = c1 * z; Y[3] = -c1 * x;
    Y[4] = c2a * x * y; Y[5] = -c2a * y * z; Y[6] = c2b * (2 * zz - xx - yy); Y[7] = -c2a * x * z; Y[8] = c2c * (xx - yy);
    Y[9] = -c3a * y * (3 * xx - yy); Y[10] = c3b * x * y * z; Y[11] = -c3c * y * (4 * zz - xx - yy);
    Y[12] = c3d * z * (2 * zz - 3 * xx - 3 * yy); Y[13] = -c3c * x * (4 * zz - xx - yy);
    Y[14] = c3e * z * (xx - yy); Y[15] = -c3a * x * (xx - 3 * yy);
}

// Gradient of each basis function with respect to (x, y, z) (treating them as independent).
void sh_basis_grad(double x, double y, double z, double dY[16][3]) {
    const double c1 = std::sqrt(3.0 / (4 * PI));
    const double c2a = std::sqrt(15.0 / (4 * PI)), c2b = std::sqrt(5.0 / (16 * PI)), c2c = std::sqrt(15.0 / (16 * PI));
    const double c3a = std::sqrt(35.0 / (32 * PI)), c3b = std::sqrt(105.0 / (4 * PI)), c3c = std::sqrt(21.0 / (32 * PI));
    const double c3d = std::sqrt(7.0 / (16 * PI)), c3e = std::sqrt(105.0 / (16 * PI));
    double xx = x * x, yy = y * y, zz = z * z;
    for (int k = 0; k < 16; ++k) dY[k][0] = dY[k][1] = dY[k][2] = 0;
    dY[1][1] = -c1; dY[2][2] = c1; dY[3][0] = -c1;
    dY[4][0] = c2a * y; dY[4][1] = c2a * x;
    dY[5][1] = -c2a * z; dY[5][2] = -c2a * y;
    dY[6][0] = -2 * c2b * x; dY[6][1] = -2 * c2b * y; dY[6][2] = 4 * c2b * z;
    dY[7][0] = -c2a * z; dY[7][2] = -c2a * x;
    dY[8][0] = 2 * c2c * x; dY[8][1] = -2 * c2c * y;
    dY[9][0] = -c3a * 6 * x * y; dY[9][1] = -c3a * (3 * xx - 3 * yy);
    dY[10][0] = c3b * y * z; dY[10][1] = c3b * x * z; dY[10][2] = c3b * x * y;
    dY[11][0] = c3c * 2 * x * y; dY[11][1] = -c3c * (4 * zz - xx - 3 * yy); dY[11][2] = -c3c * 8 * y * z;
    dY[12][0] = -c3d * 6 * x * z; dY[12][1] = -c3d * 6 * y * z; dY[12][2] = c3d * (6 * zz - 3 * xx - 3 * yy);
    dY[13][0] = -c3c * (4 * zz - 3 * xx - yy); dY[13][1] = c3c * 2 * x * y; dY[13][2] = -c3c * 8 * x * z;
    dY[14][0] = 2 * c3e * z * x; dY[14][1] = -2 * c3e * z * y; dY[14][2] = c3e * (xx - yy);
    dY[15][0] = -c3a * (3 * xx - 3 * yy); dY[15][1] = c3a * 6 * x * y;
}

// One splat, fp32 decision track.  rec: u v ca cb | cc on op t | (colour slots unused) | invK
// where (ca, cb, cc) are the conic pre-scaled so that the exponent in base 2 is
//   p2 = ca dx^2 + cb dx dy + cc dy^2.
struct SplatF { float u, v, ca, cb, cc, on, op, t, K; float depth; int32_t rect[4]; bool visible; };

const float KH = -0.72134752044448170f;   // -0.5 * log2(e), rounded to fp32
const float KL = 1.44269504088896341f;    //  log2(e), rounded to fp32

// Camera-space point of the decision track, x_c = R m + T per row as a compensated dot product
// (Dot2 of Ogita, Rump & Oishi 2005): each product is split exactly into p + e with an FMA
// (e = fmaf(a, b, -p)), partial sums are split exactly by Knuth's TwoSum, and the collected
// errors are added back at the end.  The terms enter in the order R_i0 m_0, R_i1 m_1, R_i2 m_2,
// T_i.  A plain fp32 dot product would lose the metre-scale camera-space coordinates of a
// kilometre-scale scene to cancellation between R m and T; this one is as accurate as if it had
// been evaluated in double the precision and rounded.
float dot2_f(const float* r, float t, const float m[3]) {
    auto twosum = [](float a, float b, float& err) {
        const float x = a + b;
        const float bv = x - a;
        err = (a - (x - bv)) + (b - bv);
        return x;
    };
    float acc = r[0] * m[0];
    float comp = fmaf(r[0], m[0], -acc);
    for (int j = 1; j < 3; ++j) {
        const float prod = r[j] * m[j];
        const float perr = fmaf(r[j], m[j], -prod);
        float serr;
        acc = twosum(acc, prod, serr);
        comp = comp + (serr + perr);
    }
    float serr;
    acc = twosum(acc, t, serr);
    comp = comp + serr;
    return acc + comp;
}

// x_c of cut node n with parent weight t: the node's and the parent's means mapped to camera space
// (dot2_f) and interpolated there, xc = fmaf(t, x_p, (1 - t) x_n) -- the same point as the
// transform of the interpolated mean, without rounding the km-scale interpolated mean to fp32.
void view_point_f(const OrCamera& cam, const OrHier32& h, int64_t n, float t, float xc[3]) {
    const int32_t p = h.parent[n];
    const bool use_p = (t != 0.0f) && p >= 0;
    for (int i = 0; i < 3; ++i) {
        const float xn = dot2_f(cam.R + 3 * i, cam.T[i], h.mean + 3 * n);
        if (!use_p) { xc[i] = xn; continue; }
        const float xp = dot2_f(cam.R + 3 * i, cam.T[i], h.mean + 3 * (int64_t)p);
        xc[i] = fmaf(t, xp, (1.0f - t) * xn);
    }
}

SplatF project_f(const OrCamera& cam, const OrOpts& o, const float a[NINTERP], const float xc[3]) {
    SplatF s{};
    s.visible = false;
    const float* W = cam.R;
    const float z = xc[2];
    if (!(z > cam.znear)) return s;
    const float xz = xc[0] / z, yz = xc[1] / z;
    s.u = fmaf(cam.fx, xz, cam.cx);
    s.v = fmaf(cam.fy, yz, cam.cy);
    const float limx = (0.65f * (float)cam.width) / cam.fx;
    const float limy = (0.65f * (float)cam.height) / cam.fy;
    const float txc = std::min(std::max(xz, -limx), limx);
    const float tyc = std::min(std::max(yz, -limy), limy);
    const float j00 = cam.fx / z, j11 = cam.fy / z;
    const float j02 = -(j00 * txc), j12 = -(j11 * tyc);
    // rotation of the interpolated quaternion (already unit length)
    const float qw = a[6], qx = a[7], qy = a[8], qz = a[9];
    const float xx = qx * qx, yy = qy * qy, zz = qz * qz;
    const float xy = qx * qy, xz2 = qx * qz, yz2 = qy * qz, wx = qw * qx, wy = qw * qy, wz = qw * qz;
    float Rq[3][3];
    Rq[0][0] = 1.0f - 2.0f * (yy + zz); Rq[0][1] = 2.0f * (xy - wz);        Rq[0][2] = 2.0f * (xz2 + wy);
    Rq[1][0] = 2.0f * (xy + wz);        Rq[1][1] = 1.0f - 2.0f * (xx + zz); Rq[1][2] = 2.0f * (yz2 - wx);
    Rq[2][0] = 2.0f * (xz2 - wy);       Rq[2][1] = 2.0f * (yz2 + wx);       Rq[2][2] = 1.0f - 2.0f * (xx + yy);
    // A2 = J W (2x3), then M = A2 Rq diag(s)
    float A2[2][3];
    for (int j = 0; j < 3; ++j) {
        A2[0][j] = fmaf(j02, W[6 + j], j00 * W[0 + j]);
        A2[1][j] = fmaf(j12, W[6 + j], j11 * W[3 + j]);
    }
    float M[2][3];
    for (int i = 0; i < 2; ++i)
        for (int k = 0; k < 3; ++k) {
            float acc = A2[i][0] * Rq[0][k];
            acc = fmaf(A2[i][1], Rq[1][k], acc);
            acc = fmaf(A2[i][2], Rq[2][k], acc);
            M[i][k] = acc * a[3 + k];
        }
    float ca2 = M[0][0] * M[0][0]; ca2 = fmaf(M[0][1], M[0][1], ca2); ca2 = fmaf(M[0][2], M[0][2], ca2);
    float cc2 = M[1][0] * M[1][0]; cc2 = fmaf(M[1][1], M[1][1], cc2); cc2 = fmaf(M[1][2], M[1][2], cc2);
    float cb2 = M[0][0] * M[1][0]; cb2 = fmaf(M[0][1], M[1][1], cb2); cb2 = fmaf(M[0][2], M[1][2], cb2);
    // det of the unfiltered 2D covariance as the squared norm of the cross product of M's rows
    const float k0 = fmaf(M[0][1], M[1][2], -(M[0][2] * M[1][1]));
    const float k1 = fmaf(M[0][2], M[1][0], -(M[0][0] * M[1][2]));
    const float k2 = fmaf(M[0][0], M[1][1], -(M[0][1] * M[1][0]));
    float det = k0 * k0; det = fmaf(k1, k1, det); det = fmaf(k2, k2, det);
    const float lp = o.lowpass;
    const float af = ca2 + lp, cf = cc2 + lp;
    const float detf = fmaf(lp, (ca2 + cc2) + lp, det);
    if (!(detf > 0.0f)) return s;
    const float comp = o.aa_compensate ? std::sqrt(std::max(0.0f, det / detf)) : 1.0f;
    s.ca = (cf / detf) * KH;
    s.cc = (af / detf) * KH;
    s.cb = (cb2 / detf) * KL;
    const float hm = 0.5f * (af + cf);
    const float hd = 0.5f * (af - cf);
    const float disc = std::sqrt(fmaf(hd, hd, cb2 * cb2));
    const float lmax = hm + disc;
    const float r = std::ceil(3.0f * std::sqrt(lmax));
    const int TX = (cam.width + o.tile_w - 1) / o.tile_w, TY = (cam.height + o.tile_h - 1) / o.tile_h;
    const float fx0 = std::floor((s.u - r) / (float)o.tile_w), fx1 = std::floor((s.u + r) / (float)o.tile_w);
    const float fy0 = std::floor((s.v - r) / (float)o.tile_h), fy1 = std::floor((s.v + r) / (float)o.tile_h);
    if (!(fx1 >= 0.0f && fx0 <= (float)(TX - 1) && fy1 >= 0.0f && fy0 <= (float)(TY - 1))) return s;
    s.rect[0] = (int32_t)std::max(fx0, 0.0f);
    s.rect[1] = (int32_t)std::min(fx1, (float)(TX - 1));
    s.rect[2] = (int32_t)std::max(fy0, 0.0f);
    s.rect[3] = (int32_t)std::min(fy1, (float)(TY - 1));
    s.on = a[58] * comp;
    s.op = a[59] * comp;
    s.t = a[60];
    s.K = a[61];
    s.depth = z;
    s.visible = true;
    return s;
}

// One splat, fp64 value track: natural-exponent conic (A, B, C), opacities, colour.
struct SplatD { double u, v, A, B, C, on, op, t, K, rgb[3], z; bool clamped[3]; };

SplatD project_d(const OrCamera& cam, const OrOpts& o, const double a[NINTERP]) {
    SplatD s{};
    double W[9], T[3];
    for (int i = 0; i < 9; ++i) W[i] = cam.R[i];
    for (int i = 0; i < 3; ++i) T[i] = cam.T[i];
    double xc[3];
    for (int i = 0; i < 3; ++i) xc[i] = W[3 * i] * a[0] + W[3 * i + 1] * a[1] + W[3 * i + 2] * a[2] + T[i];
    double z = xc[2];
    s.z = z;
    double xz = xc[0] / z, yz = xc[1] / z;
    s.u = (double)cam.fx * xz + cam.cx;
    s.v = (double)cam.fy * yz + cam.cy;
    double limx = 0.65 * cam.width / cam.fx, limy = 0.65 * cam.height / cam.fy;
    double txc = std::min(std::max(xz, -limx), limx), tyc = std::min(std::max(yz, -limy), limy);
    double J[2][3] = {{cam.fx / z, 0, -cam.fx * txc / z}, {0, cam.fy / z, -cam.fy * tyc / z}};
    M3 Rq = quat_to_mat(a + 6);
    double M[2][3];
    for (int i = 0; i < 2; ++i)
        for (int k = 0; k < 3; ++k) {
            double acc = 0;
            for (int j = 0; j < 3; ++j) {
                double jw = 0;
                for (int l = 0; l < 3; ++l) jw += J[i][l] * W[3 * l + j];
                acc += jw * Rq.a[j][k];
            }
            M[i][k] = acc * a[3 + k];
        }
    double aa = 0, bb = 0, cc = 0;
    for (int k = 0; k < 3; ++k) { aa += M[0][k] * M[0][k]; bb += M[0][k] * M[1][k]; cc += M[1][k] * M[1][k]; }
    double k0 = M[0][1] * M[1][2] - M[0][2] * M[1][1];
    double k1 = M[0][2] * M[1][0] - M[0][0] * M[1][2];
    double k2 = M[0][0] * M[1][1] - M[0][1] * M[1][0];
    double det = k0 * k0 + k1 * k1 + k2 * k2;
    double lp = o.lowpass;
    double af = aa + lp, cf = cc + lp, detf = af * cf - bb * bb;
    double comp = o.aa_compensate ? std::sqrt(std::max(0.0, det / detf)) : 1.0;
    s.A = cf / detf; s.B = -bb / detf; s.C = af / detf;
    s.on = a[58] * comp; s.op = a[59] * comp; s.t = a[60]; s.K = a[61];
    // view-dependent colour (SH degree 3), direction from the camera centre to the mean
    double c[3];
    for (int j = 0; j < 3; ++j) c[j] = -(W[j] * T[0] + W[3 + j] * T[1] + W[6 + j] * T[2]);
    double d[3] = {a[0] - c[0], a[1] - c[1], a[2] - c[2]};
    double dn = std::sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    double Y[16];
    sh_basis(d[0] / dn, d[1] / dn, d[2] / dn, Y);
    for (int ch = 0; ch < 3; ++ch) {
        double acc = 0.5;
        for (int k = 0; k < 16; ++k) acc += a[10 + 3 * k + ch] * Y[k];
        s.clamped[ch] = acc < 0;
        s.rgb[ch] = std::max(acc, 0.0);
    }
    return s;
}

}  // namespace

extern "C" {

// Interpolated attributes of every cut node, both tracks, SoA [62][M].
void or_interpolate(const OrHier32* h, const OrHier64* hd, int64_t M, const int32_t* ids, const float* t,
                    float* out32, double* out64) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < M; ++i) {
        float a[NINTERP];
        double b[NINTERP];
        interp_f(*h, ids[i], t[i], a);
        interp_d(*h, *hd, ids[i], (double)t[i], b);
        for (int k = 0; k < NINTERP; ++k) {
            if (out32) out32[k * M + i] = a[k];
            if (out64) out64[k * M + i] = b[k];
        }
    }
}

// Splat records of every cut node.
//   rec32 [M][10]: u v ca cb cc on op t K depth   (fp32 decision track)
//   rect  [M][4] : x0 x1 y0 y1 (tiles, inclusive), all -1 if culled
//   val64 [M][13]: u v A B C on op t K r g b z     (fp64 value track; z = view depth of the mean)
void or_preprocess(const OrCamera* cam, const OrOpts* o, const OrHier32* h, const OrHier64* hd, int64_t M,
                   const int32_t* ids, const float* t, float* rec32, int32_t* rect, double* val64) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < M; ++i) {
        float a[NINTERP];
        double b[NINTERP];
        float ti = o->interpolate ? t[i] : 0.0f;
        interp_f(*h, ids[i], ti, a);
        interp_d(*h, *hd, ids[i], (double)ti, b);
        float xc[3];
        view_point_f(*cam, *h, ids[i], ti, xc);
        SplatF sf = project_f(*cam, *o, a, xc);
        float* r = rec32 + 10 * i;
        int32_t* rc = rect + 4 * i;
        if (!sf.visible) {
            for (int k = 0; k < 10; ++k) r[k] = 0;
            rc[0] = rc[1] = rc[2] = rc[3] = -1;
            for (int k = 0; k < NVAL; ++k) val64[NVAL * i + k] = 0;
            continue;
        }
        r[0] = sf.u; r[1] = sf.v; r[2] = sf.ca; r[3] = sf.cb; r[4] = sf.cc;
        r[5] = sf.on; r[6] = sf.op; r[7] = sf.t; r[8] = sf.K; r[9] = sf.depth;
        for (int k = 0; k < 4; ++k) rc[k] = sf.rect[k];
        SplatD sd = project_d(*cam, *o, b);
        double* v = val64 + NVAL * i;
        v[0] = sd.u; v[1] = sd.v; v[2] = sd.A; v[3] = sd.B; v[4] = sd.C; v[5] = sd.on; v[6] = sd.op;
        v[7] = sd.t; v[8] = sd.K; v[9] = sd.rgb[0]; v[10] = sd.rgb[1]; v[11] = sd.rgb[2]; v[12] = sd.z;
    }
}

// Per-tile lists: every visible splat whose tile rectangle covers the tile, ordered by
// (fp32 depth ascending, cut position ascending).  ranges [n_tiles][2] = [start, end) into list.
// Returns the total number of (tile, splat) pairs (only the first cap are written).
int64_t or_tile_lists(const OrCamera* cam, const OrOpts* o, int64_t M, const float* rec32, const int32_t* rect,
                      int32_t* ranges, int32_t* list, int64_t cap) {
    const int TX = (cam->width + o->tile_w - 1) / o->tile_w, TY = (cam->height + o->tile_h - 1) / o->tile_h;
    std::vector<std::vector<int32_t>> per(TX * TY);
    for (int64_t i = 0; i < M; ++i) {
        const int32_t* rc = rect + 4 * i;
        if (rc[0] < 0) continue;
        for (int ty = rc[2]; ty <= rc[3]; ++ty)
            for (int tx = rc[0]; tx <= rc[1]; ++tx) per[ty * TX + tx].push_back((int32_t)i);
    }
    int64_t off = 0;
    for (int tile = 0; tile < TX * TY; ++tile) {
        auto& L = per[tile];
        std::stable_sort(L.begin(), L.end(), [&](int32_t a, int32_t b) { return rec32[10 * a + 9] < rec32[10 * b + 9]; });
        ranges[2 * tile] = (int32_t)off;
        for (int32_t s : L) { if (off < cap) list[off] = s; ++off; }
        ranges[2 * tile + 1] = (int32_t)off;
    }
    return off;
}

}  // extern "C"

// ==========================================================================================
// Blending (Sec. 3.1 Eq. alpha; transition opacity Eq. alphap with K children, Sec. 5.2)
// ==========================================================================================

namespace {

struct PixelRec { int32_t k; double alpha, T; };   // a contributing splat (list position, alpha, T before)

// Per-pixel fp32 decision values for one (pixel, splat) pair.  Returns alpha32.
float alpha_f(const float* r, float px, float py, float clampv) {
    const float dx = px - r[0], dy = py - r[1];
    const float h = fmaf(r[2], dx, r[3] * dy);
    const float g = (r[4] * dy) * dy;
    const float p2 = fmaf(dx, h, g);
    const float G = (float)std::exp2((double)p2);
    const float an = std::min(clampv, r[5] * G);
    const float t = r[7];
    if (t == 0.0f) return an;
    const float ap = std::min(clampv, r[6] * G);
    const float apr = (float)(1.0 - std::pow(1.0 - (double)ap, 1.0 / (double)r[8]));
    return fmaf(t, apr, (1.0f - t) * an);
}

double alpha_d(const double* v, double px, double py, double clamp, bool* cn = nullptr, bool* cp = nullptr) {
    double dx = px - v[0], dy = py - v[1];
    double pw = -0.5 * (v[2] * dx * dx + v[4] * dy * dy) - v[3] * dx * dy;
    double G = std::exp(pw);
    double xn = v[5] * G, an = std::min(clamp, xn);
    if (cn) *cn = xn >= clamp;
    double t = v[7];
    if (t == 0.0) return an;
    double xp = v[6] * G, ap = std::min(clamp, xp);
    if (cp) *cp = xp >= clamp;
    double apr = 1.0 - std::pow(1.0 - ap, 1.0 / v[8]);
    return (1.0 - t) * an + t * apr;
}

// Blend one pixel over an ordered list of splat indices.  Decisions (skip below the alpha floor,
// stop when the transmittance would fall below t_min) are taken in the fp32 track; the colour is
// accumulated in the fp64 track, and so is the expected depth sum(T alpha z) of the depth
// regulariser (the splat's colour replaced by the view depth of its mean; no background term).
// Returns the list position just after the last contributing splat (0 if none contributed).
int32_t blend_pixel(const OrOpts& o, const float* rec32, const double* val64, const int32_t* L, int32_t n,
                    double px, double py, double out[3], double& depth, double& Tfin, bool& ambiguous,
                    std::vector<PixelRec>* contrib) {
    const float pxf = (float)px, pyf = (float)py;
    const float afl = o.alpha_floor, tmin = o.t_min;
    float T32 = 1.0f;
    double T = 1.0, C[3] = {0, 0, 0}, D = 0.0;
    int32_t last = 0;
    ambiguous = false;
    for (int32_t k = 0; k < n; ++k) {
        const int32_t s = L[k];
        const float a32 = alpha_f(rec32 + 10 * s, pxf, pyf, o.alpha_clamp);
        if (std::fabs(a32 - afl) <= 1e-5f * afl) ambiguous = true;
        if (a32 < afl) continue;
        const float Tn32 = T32 * (1.0f - a32);
        if (std::fabs(Tn32 - tmin) <= 1e-5f * tmin) ambiguous = true;
        if (Tn32 < tmin) break;
        last = k + 1;
        const double* v = val64 + NVAL * s;
        double a = alpha_d(v, px, py, (double)o.alpha_clamp);
        if (contrib) contrib->push_back({k, a, T});
        for (int ch = 0; ch < 3; ++ch) C[ch] += v[9 + ch] * a * T;
        D += v[12] * a * T;
        T *= (1.0 - a);
        T32 = Tn32;
    }
    for (int ch = 0; ch < 3; ++ch) out[ch] = C[ch] + T * (double)o.bg[ch];
    depth = D;
    Tfin = T;
    return last;
}

// Exposure compensation (appendix, exposure optimisation): the camera's 3x4 affine E (row-major)
// applied to the rendered colour, out = E [C | 1].  E = NULL: the identity.
void expose(const float* E, const double in[3], double out[3]) {
    for (int c = 0; c < 3; ++c)
        out[c] = E ? (double)E[4 * c] * in[0] + (double)E[4 * c + 1] * in[1] + (double)E[4 * c + 2] * in[2]
                         + (double)E[4 * c + 3]
                   : in[c];
}

}  // namespace

extern "C" {

// Tiled blend: image [3][H][W] (fp64, exposure applied when E is given), expected depth [H][W]
// (nullable), final transmittance, the list position after the last contributing splat per pixel,
// and a per-pixel flag for decisions that fell within the fp32 ambiguity band.
void or_blend(const OrCamera* cam, const OrOpts* o, const float* rec32, const double* val64,
              const int32_t* ranges, const int32_t* list, const float* E, double* image, double* depth,
              double* T_final, int32_t* n_contrib, uint8_t* ambiguous) {
    const int W = cam->width, H = cam->height;
    const int TX = (W + o->tile_w - 1) / o->tile_w;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t pix = 0; pix < (int64_t)W * H; ++pix) {
        int x = (int)(pix % W), y = (int)(pix / W);
        int tile = (y / o->tile_h) * TX + (x / o->tile_w);
        int32_t s = ranges[2 * tile], e = ranges[2 * tile + 1];
        double out[3], ex[3], D, Tf;
        bool amb;
        int32_t c = blend_pixel(*o, rec32, val64, list + s, e - s, x + 0.5, y + 0.5, out, D, Tf, amb, nullptr);
        expose(E, out, ex);
        for (int ch = 0; ch < 3; ++ch) image[(int64_t)ch * W * H + pix] = ex[ch];
        if (depth) depth[pix] = D;
        if (T_final) T_final[pix] = Tf;
        if (n_contrib) n_contrib[pix] = c;
        if (ambiguous) ambiguous[pix] = amb;
    }
}

// Brute force without tile lists: for every pixel, gather every visible splat whose tile
// rectangle contains the pixel's tile, order by (fp32 depth, cut position), blend.
void or_blend_bruteforce(const OrCamera* cam, const OrOpts* o, int64_t M, const float* rec32, const int32_t* rect,
                         const double* val64, double* image) {
    const int W = cam->width, H = cam->height;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t pix = 0; pix < (int64_t)W * H; ++pix) {
        int x = (int)(pix % W), y = (int)(pix / W);
        int tx = x / o->tile_w, ty = y / o->tile_h;
        std::vector<int32_t> L;
        for (int64_t i = 0; i < M; ++i) {
            const int32_t* rc = rect + 4 * i;
            if (rc[0] >= 0 && tx >= rc[0] && tx <= rc[1] && ty >= rc[2] && ty <= rc[3]) L.push_back((int32_t)i);
        }
        std::sort(L.begin(), L.end(), [&](int32_t a, int32_t b) {
            float da = rec32[10 * a + 9], db = rec32[10 * b + 9];
            return da < db || (da == db && a < b);
        });
        double out[3], D, Tf;
        bool amb;
        blend_pixel(*o, rec32, val64, L.data(), (int32_t)L.size(), x + 0.5, y + 0.5, out, D, Tf, amb, nullptr);
        for (int ch = 0; ch < 3; ++ch) image[(int64_t)ch * W * H + pix] = out[ch];
    }
}

}  // extern "C"

// ==========================================================================================
// Adjoint (hierarchy optimisation, Sec. 5.1; manual alpha' derivative Sec. 7.1, clamp rule Sec. 7.3)
// ==========================================================================================

namespace {

// Per-splat gradient accumulator of the value-track parameters.
struct SplatGrad { double u, v, A, B, C, on, op, rgb[3], z; };

// Backward of the interpolation + projection of one splat: from the splat-parameter gradient to
// the interpolated attributes (mean 3, scale 3, rot 4 (pre-normalisation), sh 48, o_n, o_p).
void project_backward(const OrCamera& cam, const OrOpts& o, const double a[NINTERP], const SplatD& sd,
                      const SplatGrad& g, double da[NINTERP]) {
    for (int k = 0; k < NINTERP; ++k) da[k] = 0;
    double W[9], T[3];
    for (int i = 0; i < 9; ++i) W[i] = cam.R[i];
    for (int i = 0; i < 3; ++i) T[i] = cam.T[i];
    // ---- recompute the forward
    double xc[3];
    for (int i = 0; i < 3; ++i) xc[i] = W[3 * i] * a[0] + W[3 * i + 1] * a[1] + W[3 * i + 2] * a[2] + T[i];
    const double z = xc[2], xz = xc[0] / z, yz = xc[1] / z;
    const double fx = cam.fx, fy = cam.fy;
    const double limx = 0.65 * cam.width / cam.fx, limy = 0.65 * cam.height / cam.fy;
    const bool cx_in = xz > -limx && xz < limx, cy_in = yz > -limy && yz < limy;
    const double txc = std::min(std::max(xz, -limx), limx), tyc = std::min(std::max(yz, -limy), limy);
    double J[2][3] = {{fx / z, 0, -fx * txc / z}, {0, fy / z, -fy * tyc / z}};
    double A2[2][3];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 3; ++j) { A2[i][j] = 0; for (int l = 0; l < 3; ++l) A2[i][j] += J[i][l] * W[3 * l + j]; }
    const double* q = a + 6;
    M3 Rq = quat_to_mat(q);
    double B[2][3], M[2][3];
    for (int i = 0; i < 2; ++i)
        for (int k = 0; k < 3; ++k) {
            B[i][k] = 0;
            for (int j = 0; j < 3; ++j) B[i][k] += A2[i][j] * Rq.a[j][k];
            M[i][k] = B[i][k] * a[3 + k];
        }
    double aa = 0, bb = 0, cc = 0;
    for (int k = 0; k < 3; ++k) { aa += M[0][k] * M[0][k]; bb += M[0][k] * M[1][k]; cc += M[1][k] * M[1][k]; }
    double k0 = M[0][1] * M[1][2] - M[0][2] * M[1][1];
    double k1 = M[0][2] * M[1][0] - M[0][0] * M[1][2];
    double k2 = M[0][0] * M[1][1] - M[0][1] * M[1][0];
    const double det = k0 * k0 + k1 * k1 + k2 * k2;
    const double lp = o.lowpass;
    const double af = aa + lp, cf = cc + lp, D = af * cf - bb * bb;
    const double comp = o.aa_compensate ? std::sqrt(std::max(0.0, det / D)) : 1.0;
    // ---- opacities: on' = o_n comp, op' = o_p comp
    da[58] = g.on * comp;
    da[59] = g.op * comp;
    const double dcomp = g.on * a[58] + g.op * a[59];
    // ---- conic (A, B, C) = (cf, -bb, af) / D
    double dD = -(g.A * cf - g.B * bb + g.C * af) / (D * D);
    double dcf = g.A / D, daf = g.C / D, dbb = -g.B / D;
    double ddet = 0;
    if (o.aa_compensate && comp > 0) {
        // comp = sqrt(det / D)
        ddet += dcomp / (2 * comp * D);
        dD += -dcomp * comp / (2 * D);
    }
    daf += dD * cf; dcf += dD * af; dbb += dD * (-2 * bb);
    // det = |M0 x M1|^2 equals aa*cc - bb^2; differentiate through (aa, bb, cc)
    double daa = daf + ddet * cc, dcc = dcf + ddet * aa;
    dbb += ddet * (-2 * bb);
    double dM[2][3];
    for (int k = 0; k < 3; ++k) {
        dM[0][k] = 2 * daa * M[0][k] + dbb * M[1][k];
        dM[1][k] = 2 * dcc * M[1][k] + dbb * M[0][k];
    }
    // M = B diag(s), B = A2 Rq
    double dB[2][3];
    for (int k = 0; k < 3; ++k) {
        da[3 + k] = dM[0][k] * B[0][k] + dM[1][k] * B[1][k];
        dB[0][k] = dM[0][k] * a[3 + k];
        dB[1][k] = dM[1][k] * a[3 + k];
    }
    double dRq[3][3], dA2[2][3];
    for (int j = 0; j < 3; ++j)
        for (int k = 0; k < 3; ++k) dRq[j][k] = A2[0][j] * dB[0][k] + A2[1][j] * dB[1][k];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 3; ++j) { dA2[i][j] = 0; for (int k = 0; k < 3; ++k) dA2[i][j] += dB[i][k] * Rq.a[j][k]; }
    double dJ[2][3];
    for (int i = 0; i < 2; ++i)
        for (int l = 0; l < 3; ++l) { dJ[i][l] = 0; for (int j = 0; j < 3; ++j) dJ[i][l] += dA2[i][j] * W[3 * l + j]; }
    // J entries: fx/z, -fx txc / z, fy/z, -fy tyc / z
    double dz = dJ[0][0] * (-fx / (z * z)) + dJ[0][2] * (fx * txc / (z * z))
              + dJ[1][1] * (-fy / (z * z)) + dJ[1][2] * (fy * tyc / (z * z));
    double dtxc = dJ[0][2] * (-fx / z), dtyc = dJ[1][2] * (-fy / z);
    double dxz = g.u * fx + (cx_in ? dtxc : 0.0);
    double dyz = g.v * fy + (cy_in ? dtyc : 0.0);
    // g.z: the expected-depth channel reads the view depth z = xc[2] directly
    double dxc[3] = {dxz / z, dyz / z, dz + g.z - dxz * xc[0] / (z * z) - dyz * xc[1] / (z * z)};
    for (int j = 0; j < 3; ++j) da[j] = W[j] * dxc[0] + W[3 + j] * dxc[1] + W[6 + j] * dxc[2];
    // rotation matrix of the (unit) quaternion w.r.t. its components
    const double w = q[0], x = q[1], y = q[2], zq = q[3];
    double dqn[4];
    dqn[0] = 2 * (-zq * dRq[0][1] + y * dRq[0][2] + zq * dRq[1][0] - x * dRq[1][2] - y * dRq[2][0] + x * dRq[2][1]);
    dqn[1] = 2 * (y * dRq[0][1] + zq * dRq[0][2] + y * dRq[1][0] - 2 * x * dRq[1][1] - w * dRq[1][2]
                  + zq * dRq[2][0] + w * dRq[2][1] - 2 * x * dRq[2][2]);
    dqn[2] = 2 * (-2 * y * dRq[0][0] + x * dRq[0][1] + w * dRq[0][2] + x * dRq[1][0] + zq * dRq[1][2]
                  - w * dRq[2][0] + zq * dRq[2][1] - 2 * y * dRq[2][2]);
    dqn[3] = 2 * (-2 * zq * dRq[0][0] - w * dRq[0][1] + x * dRq[0][2] + w * dRq[1][0] - 2 * zq * dRq[1][1]
                  + y * dRq[1][2] + x * dRq[2][0] + y * dRq[2][1]);
    for (int k = 0; k < 4; ++k) da[6 + k] = dqn[k];   // w.r.t. the normalised quaternion (caller maps back)
    // colour: rgb = max(0, sum sh Y(dir) + 0.5), dir = (mean - c) / |mean - c|
    double c[3];
    for (int j = 0; j < 3; ++j) c[j] = -(W[j] * T[0] + W[3 + j] * T[1] + W[6 + j] * T[2]);
    double d[3] = {a[0] - c[0], a[1] - c[1], a[2] - c[2]};
    double dn = std::sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    double u3[3] = {d[0] / dn, d[1] / dn, d[2] / dn};
    double Y[16], dY[16][3];
    sh_basis(u3[0], u3[1], u3[2], Y);
    sh_basis_grad(u3[0], u3[1], u3[2], dY);
    double ddir[3] = {0, 0, 0};
    for (int ch = 0; ch < 3; ++ch) {
        if (sd.clamped[ch]) continue;
        for (int k = 0; k < 16; ++k) {
            da[10 + 3 * k + ch] = g.rgb[ch] * Y[k];
            for (int j = 0; j < 3; ++j) ddir[j] += g.rgb[ch] * a[10 + 3 * k + ch] * dY[k][j];
        }
    }
    double dot = ddir[0] * u3[0] + ddir[1] * u3[1] + ddir[2] * u3[2];
    for (int j = 0; j < 3; ++j) da[j] += (ddir[j] - u3[j] * dot) / dn;
}

}  // namespace

extern "C" {

// Gradient of L = sum(dL_dimage * image) + sum(dL_ddepth * depth) w.r.t. the value-track node
// attributes (image with the camera's exposure E applied when given; dL_ddepth nullable).
// grad [N][59] (mean 3, scale 3, rot 4, opacity 1, sh 48) is OVERWRITTEN.  Node n receives
// (1 - t) of its interpolated attributes' gradient and the parent p receives t of it (t is a
// constant); o_n and o_p receive the gradients of their own opacity terms; the opacity gradient
// of a branch is zero where that branch's alpha is clamped.  freeze_leaves zeroes leaf rows.
void or_backward(const OrCamera* cam, const OrOpts* o, const OrHier32* h, const OrHier64* hd, int64_t M,
                 const int32_t* ids, const float* t, const float* rec32, const int32_t* rect, const double* val64,
                 const int32_t* ranges,
                 const int32_t* list, const double* dL_dimage, const double* dL_ddepth, const float* E,
                 int32_t freeze_leaves, double* grad) {
    const int Wd = cam->width, Ht = cam->height;
    const int TX = (Wd + o->tile_w - 1) / o->tile_w, TY = (Ht + o->tile_h - 1) / o->tile_h;
    const double clampv = o->alpha_clamp;
    int nthreads = 1;
#ifdef _OPENMP
    nthreads = omp_get_max_threads();
#endif
    std::vector<std::vector<SplatGrad>> acc(nthreads, std::vector<SplatGrad>(M, SplatGrad{}));
#pragma omp parallel for schedule(dynamic, 1)
    for (int tile = 0; tile < TX * TY; ++tile) {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        std::vector<SplatGrad>& G = acc[tid];
        const int tx = tile % TX, ty = tile / TX;
        const int32_t* L = list + ranges[2 * tile];
        const int32_t n = ranges[2 * tile + 1] - ranges[2 * tile];
        std::vector<PixelRec> rec;
        for (int y = ty * o->tile_h; y < std::min(Ht, (ty + 1) * o->tile_h); ++y)
            for (int x = tx * o->tile_w; x < std::min(Wd, (tx + 1) * o->tile_w); ++x) {
                rec.clear();
                double out[3], D, Tf;
                bool amb;
                const double px = x + 0.5, py = y + 0.5;
                blend_pixel(*o, rec32, val64, L, n, px, py, out, D, Tf, amb, &rec);
                const int64_t pix = (int64_t)y * Wd + x;
                double gout[3], gpix[3];
                for (int ch = 0; ch < 3; ++ch) gout[ch] = dL_dimage[(int64_t)ch * Wd * Ht + pix];
                // through the exposure: dL/dC_k = sum_c E[c][k] dL/dout_c
                for (int k = 0; k < 3; ++k)
                    gpix[k] = E ? (double)E[k] * gout[0] + (double)E[4 + k] * gout[1] + (double)E[8 + k] * gout[2]
                                : gout[k];
                const double gD = dL_ddepth ? dL_ddepth[pix] : 0.0;
                // S = colour accumulated behind the current splat, plus the background term; SD the depth
                double S[3], SD = 0.0;
                for (int ch = 0; ch < 3; ++ch) S[ch] = Tf * o->bg[ch];
                for (int r = (int)rec.size() - 1; r >= 0; --r) {
                    const int32_t s = L[rec[r].k];
                    const double* v = val64 + NVAL * s;
                    const double a = rec[r].alpha, Tk = rec[r].T;
                    SplatGrad& gs = G[s];
                    double dalpha = 0;
                    for (int ch = 0; ch < 3; ++ch) {
                        gs.rgb[ch] += gpix[ch] * a * Tk;
                        dalpha += gpix[ch] * (Tk * v[9 + ch] - S[ch] / (1.0 - a));
                    }
                    gs.z += gD * a * Tk;
                    dalpha += gD * (Tk * v[12] - SD / (1.0 - a));
                    for (int ch = 0; ch < 3; ++ch) S[ch] += v[9 + ch] * a * Tk;
                    SD += v[12] * a * Tk;
                    // alpha = (1 - t) an + t a'(ap);  an = min(c, on G);  ap = min(c, op G)
                    const double dx = px - v[0], dy = py - v[1];
                    const double pw = -0.5 * (v[2] * dx * dx + v[4] * dy * dy) - v[3] * dx * dy;
                    const double Gv = std::exp(pw);
                    const double tt = v[7], K = v[8];
                    double dG = 0;
                    const double xn = v[5] * Gv;
                    const double dan = (tt == 0.0) ? dalpha : (1.0 - tt) * dalpha;
                    if (xn < clampv) { gs.on += dan * Gv; dG += dan * v[5]; }
                    if (tt != 0.0) {
                        const double xp = v[6] * Gv;
                        if (xp < clampv) {
                            const double ap = xp;
                            const double dapr_dap = (1.0 / K) * std::pow(1.0 - ap, 1.0 / K - 1.0);
                            const double dap = tt * dalpha * dapr_dap;
                            gs.op += dap * Gv;
                            dG += dap * v[6];
                        }
                    }
                    const double dpw = dG * Gv;
                    gs.A += -0.5 * dx * dx * dpw;
                    gs.C += -0.5 * dy * dy * dpw;
                    gs.B += -dx * dy * dpw;
                    gs.u += dpw * (v[2] * dx + v[3] * dy);
                    gs.v += dpw * (v[3] * dx + v[4] * dy);
                }
            }
    }
    std::vector<SplatGrad> tot(M, SplatGrad{});
    for (int th = 0; th < nthreads; ++th)
        for (int64_t s = 0; s < M; ++s) {
            const SplatGrad& a = acc[th][s];
            SplatGrad& b = tot[s];
            b.u += a.u; b.v += a.v; b.A += a.A; b.B += a.B; b.C += a.C; b.on += a.on; b.op += a.op; b.z += a.z;
            for (int ch = 0; ch < 3; ++ch) b.rgb[ch] += a.rgb[ch];
        }
    std::fill(grad, grad + (size_t)h->n * NATTR, 0.0);
    for (int64_t s = 0; s < M; ++s) {
        if (rect[4 * s] < 0) continue;  // culled: never blended
        const int64_t n = ids[s];
        const int32_t p = h->parent[n];
        const double ts = o->interpolate ? (double)t[s] : 0.0;
        double a[NINTERP], da[NINTERP];
        interp_d(*h, *hd, n, ts, a);
        SplatD sd = project_d(*cam, *o, a);
        project_backward(*cam, *o, a, sd, tot[s], da);
        // back through the quaternion normalisation: q = ql / |ql|
        double ql[4];
        for (int d = 0; d < 4; ++d)
            ql[d] = (ts != 0.0 && p >= 0) ? (1 - ts) * hd->rot[4 * n + d] + ts * hd->rot[4 * (int64_t)p + d] : hd->rot[4 * n + d];
        double nl = std::sqrt(ql[0] * ql[0] + ql[1] * ql[1] + ql[2] * ql[2] + ql[3] * ql[3]);
        double dot = 0;
        for (int d = 0; d < 4; ++d) dot += a[6 + d] * da[6 + d];
        double dql[4];
        for (int d = 0; d < 4; ++d) dql[d] = (da[6 + d] - a[6 + d] * dot) / nl;
        double* gn = grad + (size_t)n * NATTR;
        const double wn = (ts != 0.0 && p >= 0) ? 1.0 - ts : 1.0;
        for (int d = 0; d < 6; ++d) gn[d] += wn * da[d];
        for (int d = 0; d < 4; ++d) gn[6 + d] += wn * dql[d];
        gn[10] += da[58];
        for (int c = 0; c < NSH; ++c) gn[11 + c] += wn * da[10 + c];
        if (p >= 0) {
            double* gp = grad + (size_t)p * NATTR;
            gp[10] += da[59];
            if (ts != 0.0) {
                for (int d = 0; d < 6; ++d) gp[d] += ts * da[d];
                for (int d = 0; d < 4; ++d) gp[6 + d] += ts * dql[d];
                for (int c = 0; c < NSH; ++c) gp[11 + c] += ts * da[10 + c];
            }
        }
    }
    if (freeze_leaves)
        for (int64_t v = 0; v < h->n; ++v)
            if (h->child_count[v] == 0) std::fill(grad + (size_t)v * NATTR, grad + (size_t)(v + 1) * NATTR, 0.0);
}

// Loss value L = sum(w * image) + sum(w_depth * depth) of the fp64 track with fixed decisions (for
// finite differences); E and w_depth nullable.
double or_weighted_image_sum(const OrCamera* cam, const OrOpts* o, const float* rec32, const double* val64,
                             const int32_t* ranges, const int32_t* list, const float* E, const double* w,
                             const double* w_depth) {
    const int W = cam->width, H = cam->height;
    std::vector<double> img((size_t)3 * W * H), dep((size_t)W * H);
    or_blend(cam, o, rec32, val64, ranges, list, E, img.data(), dep.data(), nullptr, nullptr, nullptr);
    double s = 0;
    for (size_t i = 0; i < img.size(); ++i) s += w[i] * img[i];
    if (w_depth)
        for (size_t i = 0; i < dep.size(); ++i) s += w_depth[i] * dep[i];
    return s;
}

// The per-pixel alpha of both tracks at n (splat, pixel-centre) pairs, exposed so that the fp32
// decision track can be checked against the fp64 value track: a32[i] = alpha_f of splat s[i]'s
// record at (px[i], py[i]) (rounded to fp32 as the blend does), a64[i] = alpha_d there.
void or_pair_alpha(const float* rec32, const double* val64, int64_t n, const int32_t* s, const double* px,
                   const double* py, float clampv, float* a32, double* a64) {
    for (int64_t i = 0; i < n; ++i) {
        a32[i] = alpha_f(rec32 + 10 * (int64_t)s[i], (float)px[i], (float)py[i], clampv);
        a64[i] = alpha_d(val64 + NVAL * (int64_t)s[i], px[i], py[i], (double)clampv);
    }
}

// Ellipsoid surface area used by the merge weights (exposed for the closed-form test).
double or_ellipsoid_area(const double* s) { return ellipsoid_area(s); }

// The degree-3 real SH basis at a unit direction (exposed for the orthonormality test).
void or_sh_basis(double x, double y, double z, double* Y) { sh_basis(x, y, z, Y); }

int32_t or_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

}  // extern "C"
