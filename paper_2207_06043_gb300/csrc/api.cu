// Host runtime of libibl: context and member set-up, mesh topology and rest
// quantities, device buffers, the per-step launch sequence with CUDA-graph
// replay, read-out and the C ABI of include/ibl.h.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <utility>
#include <vector>

#include "../../include/ibl.h"
#include "ibl_internal.cuh"

using namespace ibl;

// Elements added to every population plane beyond the padded node count
// (a multiple of 32 keeps every 32-node run 128-byte aligned).
#ifndef IBL_PLANE_PAD
#define IBL_PLANE_PAD 0
#endif

namespace {

thread_local std::string g_last_error;

struct CapsuleHost {
    std::vector<double> X;
    std::vector<int> tris;
    double vel0[3] = {0, 0, 0};
    ibl_capsule_params p{};
};

struct MemberHost {
    ibl_lattice_desc desc{};
    std::vector<uint8_t> tag;
    std::vector<ibl_wall_link> links;
    int face_kind[6] = {0, 0, 0, 0, 0, 0};
    double face_rho[6] = {1, 1, 1, 1, 1, 1};
    std::vector<float> face_vel[6];
    std::vector<float> init_rho, init_u;
    std::vector<CapsuleHost> caps;
    // the whole lattice of a slab context as its capsules see it: tags and
    // capsules only, no populations, links or faces
    bool whole_view = false;
};

// Rest data of one capsule kept on the host for read-out.
struct CapsuleRestHost {
    int member, v_begin, nv, t_begin, nt, e_begin, ne;
    double S0, V0;
    std::vector<double> l0;
    std::vector<int> edges;   // 2 per edge, local vertex ids
    int rigid;
};

}  // namespace

struct ibl_ctx {
    cudaStream_t user_stream = nullptr;
    cudaStream_t work = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    cudaStream_t work2 = nullptr, work3 = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_ib = nullptr, ev_shell = nullptr, ev_probes = nullptr;
    int storage = IBL_STORAGE_F32;
    std::vector<MemberHost> members;
    bool finalized = false;
    long long t = 0;   // steps launched
    DevState dev;
    std::vector<MemberDev> hmem;
    std::vector<CapsuleRestHost> rest;
    std::vector<std::vector<int>> member_caps;   // global capsule ids per member
    std::vector<void*> allocs;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    int graph_kernels[2] = {0, 0};   // kernel nodes of each parity's step graph
    bool use_graphs = true;
    int threads = 128;   // lattice kernel block size (the compiled bound)
    int blocks_per_sm = 0;
    int lattice_path = 0;   // 1: staged lattice kernel where available, 0: register gathers
    int n_sm = 0;
    int device = -1;                   // CUDA device current when the context was created
    float* noalloc = nullptr;          // that device's copy of the static read array
    float* stage = nullptr;            // device staging buffer of host reads, kept and grown
    size_t stage_bytes = 0;
    double* cap_stats = nullptr;       // CAP_STAT_DOUBLES per capsule (ibl_read_capsules)
    std::vector<double> h_cap_stats;
    bool timing = false;
    // slab decomposition along x (ibl_slab_group_create): member m is slab m
    struct Slabs {
        int S = 0, H = 0, nx = 0, per = 0;
        std::vector<ibl_slab> sl;
    } slabs;
    std::vector<cudaEvent_t> tev;
    double ktime[4] = {0, 0, 0, 0};
    std::vector<int> h_counters;
    std::vector<uint32_t> h_status;
    std::string err;
    // adjoint work buffers and segment graphs, kept between ibl_adjoint calls
    struct AdjSeg { int kind, mode, parity, len; float* lin; int tb; cudaGraphExec_t exec; };
    struct AdjCache {
        int kind = -1;   // 0: flow objective (lattice only), 1: capsule objective
        size_t ck_bytes = 0, tape_steps = 0, tape2_steps = 0;
        char *ck = nullptr, *snap = nullptr;
        float4* tape_rhou = nullptr;
        float *tape_dvdq = nullptr, *tape_rho = nullptr, *lamA = nullptr, *lamB = nullptr;
        double* acc = nullptr;
        // capsule objective: IB-force and vertex tapes, per-vertex adjoints
        float4* tape_F = nullptr;
        double *tape_x = nullptr, *tape_v = nullptr;
        // a second tape, so that the recompute of one segment runs beside the
        // reverse sweep of the next, and the reverse sweep's own copies of the
        // geometry buffers it rebuilds at every step
        float4 *tape2_rhou = nullptr, *tape2_F = nullptr;
        float *tape2_dvdq = nullptr, *tape2_rho = nullptr;
        double *tape2_x = nullptr, *tape2_v = nullptr;
        double* rx = nullptr;
        float4 *rxm = nullptr, *rvacc = nullptr;
        float *rnrm = nullptr, *rarea = nullptr;
        CapsuleSums* rsums = nullptr;
        cudaStream_t rs = nullptr;
        cudaEvent_t ev_rec[2] = {nullptr, nullptr}, ev_rev[2] = {nullptr, nullptr}, ev_fwd = nullptr;
        AdjCapPtrs cp;
        std::vector<AdjSeg> graphs;
    } adj;
};

namespace {

ibl_status fail(ibl_ctx* ctx, ibl_status st, const std::string& msg) {
    if (ctx) ctx->err = msg;
    else g_last_error = msg;
    return st;
}

#define CK(call)                                                                               \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            return fail(ctx, IBL_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

#define CKS(call)                                   \
    do {                                            \
        ibl_status s_ = (call);                     \
        if (s_ != IBL_OK) return s_;                \
    } while (0)

// fn(begin, end) over [0, n) in up to hardware_concurrency chunks of at least
// min_chunk items, on host threads (the calling thread takes the first chunk).
template <typename F>
void parallel_chunks(size_t n, size_t min_chunk, F fn) {
    const size_t hw = std::max(1u, std::thread::hardware_concurrency());
    const size_t T = std::min(hw, std::max<size_t>(1, n / std::max<size_t>(min_chunk, 1)));
    if (T <= 1) {
        fn((size_t)0, n);
        return;
    }
    const size_t step = (n + T - 1) / T;
    std::vector<std::thread> th;
    for (size_t t = 1; t < T; ++t) {
        const size_t b = t * step, e = std::min(n, b + step);
        if (b < e) th.emplace_back([&fn, b, e] { fn(b, e); });
    }
    fn((size_t)0, std::min(n, step));
    for (std::thread& x : th) x.join();
}

template <typename T>
ibl_status dev_alloc(ibl_ctx* ctx, T*& p, size_t count) {
    p = nullptr;
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc((void**)&p, sizeof(T) * count);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, IBL_ERR_OOM, std::string("cudaMalloc of ") + std::to_string(sizeof(T) * count) +
                                          " bytes failed: " + cudaGetErrorString(e));
    }
    ctx->allocs.push_back((void*)p);
    return IBL_OK;
}

template <typename T>
ibl_status upload(ibl_ctx* ctx, T* dst, const std::vector<T>& src) {
    if (src.empty()) return IBL_OK;
    CK(cudaMemcpyAsync(dst, src.data(), sizeof(T) * src.size(), cudaMemcpyHostToDevice, ctx->work));
    return IBL_OK;
}

inline size_t round_up(size_t a, size_t b) { return (a + b - 1) / b * b; }

// ---------------------------------------------------------------------------
// mesh topology and rest quantities (Section "Deforming bodies constitutive
// model"); independent host implementation
// ---------------------------------------------------------------------------
struct V3 { double x, y, z; };
inline V3 vsub(V3 a, V3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
inline V3 vcross(V3 a, V3 b) { return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x}; }
inline double vdot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
inline double vnorm(V3 a) { return std::sqrt(vdot(a, a)); }

// hinges: for every edge {p<q}: (wing of p->q, p, q, wing of q->p), sorted by (p, q)
// Hinges of a closed, consistently oriented triangle mesh: for every edge
// u < v, the wing vertex of the triangle holding the half-edge u->v, u, v, and
// the wing of the triangle holding v->u (edges in (u, v) order).  Half-edges
// are sorted by (u, v) instead of kept in a tree: meshes of thousands of
// vertices are set up in a millisecond.
bool build_hinges(const std::vector<int>& tris, int nv, std::vector<int>& hinge, std::vector<int>& tri_a,
                  std::vector<int>& tri_b, std::string& why) {
    // half-edges u -> v (with their triangle and the triangle's third vertex)
    // bucketed by u; every edge u < v pairs with v -> u.  Edges come out in
    // ascending (u, v) order.
    const int nt = (int)tris.size() / 3;
    struct Half { int v, t, wing; };
    std::vector<int> start(nv + 1, 0);
    for (int t = 0; t < nt; ++t) {
        const int a = tris[3 * t], b = tris[3 * t + 1], c = tris[3 * t + 2];
        if (a < 0 || b < 0 || c < 0 || a >= nv || b >= nv || c >= nv || a == b || b == c || a == c) {
            why = "triangle " + std::to_string(t) + " has an invalid vertex index";
            return false;
        }
        ++start[a + 1]; ++start[b + 1]; ++start[c + 1];
    }
    for (int v = 0; v < nv; ++v) start[v + 1] += start[v];
    std::vector<Half> half(3 * (size_t)nt);
    std::vector<int> at(start.begin(), start.end() - 1);
    for (int t = 0; t < nt; ++t) {
        const int a = tris[3 * t], b = tris[3 * t + 1], c = tris[3 * t + 2];
        const int uvw[3][3] = {{a, b, c}, {b, c, a}, {c, a, b}};
        for (auto& r : uvw) half[at[r[0]]++] = {r[1], t, r[2]};
    }
    for (int u = 0; u < nv; ++u) {
        auto b = half.begin() + start[u], e = half.begin() + start[u + 1];
        std::sort(b, e, [](const Half& x, const Half& y) { return x.v < y.v; });
        for (auto it = b; it + 1 < e; ++it)
            if (it->v == (it + 1)->v) {
                why = "edge used twice in the same direction (mesh not consistently oriented)";
                return false;
            }
    }
    hinge.clear(); tri_a.clear(); tri_b.clear();
    size_t paired = 0;
    for (int u = 0; u < nv; ++u)
        for (int i = start[u]; i < start[u + 1]; ++i) {
            const Half& h = half[i];
            if (u > h.v) continue;
            const Half* back = nullptr;
            for (int k = start[h.v]; k < start[h.v + 1]; ++k)
                if (half[k].v == u) { back = &half[k]; break; }
            if (!back) { why = "mesh is not closed"; return false; }
            hinge.push_back(h.wing);
            hinge.push_back(u);
            hinge.push_back(h.v);
            hinge.push_back(back->wing);
            tri_a.push_back(h.t);
            tri_b.push_back(back->t);
            ++paired;
        }
    if (2 * paired != half.size()) { why = "mesh is not closed"; return false; }
    return true;
}

double signed_dihedral(V3 v1, V3 v2, V3 v3, V3 v4) {
    const V3 nA = vcross(vsub(v2, v1), vsub(v3, v1));
    const V3 nB = vcross(vsub(v3, v4), vsub(v2, v4));
    const V3 e = vsub(v3, v2);
    const double L = vnorm(e);
    const V3 eh = {e.x / L, e.y / L, e.z / L};
    return std::atan2(vdot(vcross(nA, nB), eh), vdot(nA, nB));
}

struct MeshSums { double V, S; V3 cen; double M2[6]; };

// volume, area, volume centroid and second moments about the centroid of a
// closed mesh (tetrahedra fanned from the vertex mean)
MeshSums mesh_sums(const double* X, int nv, const int* tris, int nt) {
    V3 o = {0, 0, 0};
    for (int v = 0; v < nv; ++v) { o.x += X[3 * v]; o.y += X[3 * v + 1]; o.z += X[3 * v + 2]; }
    o.x /= nv; o.y /= nv; o.z /= nv;
    MeshSums s{};
    double cen[3] = {0, 0, 0};
    for (int t = 0; t < nt; ++t) {
        const int* T = tris + 3 * t;
        const V3 a = vsub({X[3 * T[0]], X[3 * T[0] + 1], X[3 * T[0] + 2]}, o);
        const V3 b = vsub({X[3 * T[1]], X[3 * T[1] + 1], X[3 * T[1] + 2]}, o);
        const V3 c = vsub({X[3 * T[2]], X[3 * T[2] + 1], X[3 * T[2] + 2]}, o);
        const double v = vdot(a, vcross(b, c)) / 6.0;
        s.V += v;
        s.S += 0.5 * vnorm(vcross(vsub(b, a), vsub(c, a)));
        const V3 q = {a.x + b.x + c.x, a.y + b.y + c.y, a.z + b.z + c.z};
        cen[0] += v * q.x / 4; cen[1] += v * q.y / 4; cen[2] += v * q.z / 4;
        const double w = v / 20.0;
        s.M2[0] += w * (a.x * a.x + b.x * b.x + c.x * c.x + q.x * q.x);
        s.M2[1] += w * (a.y * a.y + b.y * b.y + c.y * c.y + q.y * q.y);
        s.M2[2] += w * (a.z * a.z + b.z * b.z + c.z * c.z + q.z * q.z);
        s.M2[3] += w * (a.x * a.y + b.x * b.y + c.x * c.y + q.x * q.y);
        s.M2[4] += w * (a.x * a.z + b.x * b.z + c.x * c.z + q.x * q.z);
        s.M2[5] += w * (a.y * a.z + b.y * b.z + c.y * c.z + q.y * q.z);
    }
    const V3 cr = {cen[0] / s.V, cen[1] / s.V, cen[2] / s.V};
    s.M2[0] -= s.V * cr.x * cr.x; s.M2[1] -= s.V * cr.y * cr.y; s.M2[2] -= s.V * cr.z * cr.z;
    s.M2[3] -= s.V * cr.x * cr.y; s.M2[4] -= s.V * cr.x * cr.z; s.M2[5] -= s.V * cr.y * cr.z;
    s.cen = {o.x + cr.x, o.y + cr.y, o.z + cr.z};
    return s;
}

// eigenvalues of a symmetric 3x3 matrix (xx yy zz xy xz yz), ascending, by
// the trigonometric solution of the characteristic cubic
void sym3_eigen(const double M[6], double ev[3]) {
    const double a00 = M[0], a11 = M[1], a22 = M[2], a01 = M[3], a02 = M[4], a12 = M[5];
    const double p1 = a01 * a01 + a02 * a02 + a12 * a12;
    const double q = (a00 + a11 + a22) / 3.0;
    const double p2 = (a00 - q) * (a00 - q) + (a11 - q) * (a11 - q) + (a22 - q) * (a22 - q) + 2.0 * p1;
    if (p2 <= 0.0) { ev[0] = ev[1] = ev[2] = q; return; }
    const double p = std::sqrt(p2 / 6.0);
    const double b00 = (a00 - q) / p, b11 = (a11 - q) / p, b22 = (a22 - q) / p;
    const double b01 = a01 / p, b02 = a02 / p, b12 = a12 / p;
    const double det = b00 * (b11 * b22 - b12 * b12) - b01 * (b01 * b22 - b12 * b02) + b02 * (b01 * b12 - b11 * b02);
    const double r = std::min(1.0, std::max(-1.0, det / 2.0));
    const double phi = std::acos(r) / 3.0;
    const double e1 = q + 2.0 * p * std::cos(phi);
    const double e3 = q + 2.0 * p * std::cos(phi + 2.0 * M_PI / 3.0);
    ev[0] = e3; ev[1] = 3.0 * q - e1 - e3; ev[2] = e1;
    std::sort(ev, ev + 3);
}

// Unit eigenvector of a symmetric 3x3 matrix (xx yy zz xy xz yz) for a simple
// eigenvalue ev: the longest cross product of two rows of M - ev I.
V3 sym3_vector(const double M[6], double ev) {
    const V3 r0 = {M[0] - ev, M[3], M[4]}, r1 = {M[3], M[1] - ev, M[5]}, r2 = {M[4], M[5], M[2] - ev};
    const V3 c[3] = {vcross(r0, r1), vcross(r0, r2), vcross(r1, r2)};
    int best = 0;
    for (int i = 1; i < 3; ++i)
        if (vdot(c[i], c[i]) > vdot(c[best], c[best])) best = i;
    const double n = vnorm(c[best]);
    return {c[best].x / n, c[best].y / n, c[best].z / n};
}

// Objective of the capsule adjoint, J = wD D + wOff y_c (D the Taylor index,
// y_c the y of the volume centroid, as ibl_read_capsule computes them from
// the tetrahedra fanned from the vertex mean o), and dJ/dx in g[3 nv], by
// reverse mode through the same sums: per triangle (a, b, c relative to o)
// v = a.(b x c)/6, q = a + b + c, V += v, S1 += v q/4,
// M2 += v/20 (a a^T + b b^T + c c^T + q q^T); C = M2 - S1 S1^T / V;
// D from the extreme eigenvalues l of C through a = sqrt(5 l / V), whose
// derivatives are v v^T (simple eigenvalues).
double capsule_objective_grad(const double* X, int nv, const int* tris, int nt, double wD, double wOff, double* g) {
    const MeshSums ms = mesh_sums(X, nv, tris, nt);
    V3 o = {0, 0, 0};
    for (int v = 0; v < nv; ++v) { o.x += X[3 * v]; o.y += X[3 * v + 1]; o.z += X[3 * v + 2]; }
    o.x /= nv; o.y /= nv; o.z /= nv;
    const double V = ms.V;
    const double S1[3] = {(ms.cen.x - o.x) * V, (ms.cen.y - o.y) * V, (ms.cen.z - o.z) * V};
    double ev[3];
    sym3_eigen(ms.M2, ev);
    const double a0 = std::sqrt(std::max(5.0 * ev[0] / V, 0.0)), a2 = std::sqrt(std::max(5.0 * ev[2] / V, 0.0));
    const double D = (a2 - a0) / (a2 + a0);
    const double J = wD * D + wOff * ms.cen.y;
    // adjoints of the extreme eigenvalues, then of C (symmetric, full)
    const double s2 = (a2 + a0) * (a2 + a0);
    const double dDa2 = 2.0 * a0 / s2, dDa0 = -2.0 * a2 / s2;
    const double lev2 = wD * dDa2 * a2 / (2.0 * ev[2]), lev0 = wD * dDa0 * a0 / (2.0 * ev[0]);
    double lV = wD * (dDa2 * (-a2 / (2.0 * V)) + dDa0 * (-a0 / (2.0 * V)));
    const V3 e2 = sym3_vector(ms.M2, ev[2]), e0 = sym3_vector(ms.M2, ev[0]);
    const double E2[3] = {e2.x, e2.y, e2.z}, E0[3] = {e0.x, e0.y, e0.z};
    double lC[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) lC[i][j] = lev2 * E2[i] * E2[j] + lev0 * E0[i] * E0[j];
    // C = M2 - S1 S1^T / V; y_c = o_y + S1_y / V
    double lS1[3];
    for (int i = 0; i < 3; ++i) {
        double t = 0.0;
        for (int j = 0; j < 3; ++j) t += lC[i][j] * S1[j];
        lS1[i] = -2.0 * t / V;
    }
    double sCs = 0.0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) sCs += S1[i] * lC[i][j] * S1[j];
    lV += sCs / (V * V);
    lS1[1] += wOff / V;
    lV += -wOff * S1[1] / (V * V);
    double lo[3] = {0.0, wOff, 0.0};
    for (int i = 0; i < 3 * nv; ++i) g[i] = 0.0;
    auto quad = [&](const double u[3], double w) {   // w lC u + w lC^T u
        V3 r;
        r.x = 2.0 * w * (lC[0][0] * u[0] + lC[0][1] * u[1] + lC[0][2] * u[2]);
        r.y = 2.0 * w * (lC[1][0] * u[0] + lC[1][1] * u[1] + lC[1][2] * u[2]);
        r.z = 2.0 * w * (lC[2][0] * u[0] + lC[2][1] * u[1] + lC[2][2] * u[2]);
        return r;
    };
    auto uqu = [&](const double u[3]) {
        double t = 0.0;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) t += u[i] * lC[i][j] * u[j];
        return t;
    };
    for (int t = 0; t < nt; ++t) {
        const int* T = tris + 3 * t;
        const double a[3] = {X[3 * T[0]] - o.x, X[3 * T[0] + 1] - o.y, X[3 * T[0] + 2] - o.z};
        const double b[3] = {X[3 * T[1]] - o.x, X[3 * T[1] + 1] - o.y, X[3 * T[1] + 2] - o.z};
        const double c[3] = {X[3 * T[2]] - o.x, X[3 * T[2] + 1] - o.y, X[3 * T[2] + 2] - o.z};
        const double q[3] = {a[0] + b[0] + c[0], a[1] + b[1] + c[1], a[2] + b[2] + c[2]};
        const V3 A = {a[0], a[1], a[2]}, B = {b[0], b[1], b[2]}, Cc = {c[0], c[1], c[2]};
        const double v = vdot(A, vcross(B, Cc)) / 6.0;
        const double lv = lV + (lS1[0] * q[0] + lS1[1] * q[1] + lS1[2] * q[2]) / 4.0 +
                          (uqu(a) + uqu(b) + uqu(c) + uqu(q)) / 20.0;
        const V3 lq = quad(q, v / 20.0);
        const double lq3[3] = {v * lS1[0] / 4.0 + lq.x, v * lS1[1] / 4.0 + lq.y, v * lS1[2] / 4.0 + lq.z};
        const V3 ga = quad(a, v / 20.0), gb = quad(b, v / 20.0), gc = quad(c, v / 20.0);
        const V3 bc = vcross(B, Cc), ca = vcross(Cc, A), ab = vcross(A, B);
        const double la[3] = {lq3[0] + ga.x + lv * bc.x / 6.0, lq3[1] + ga.y + lv * bc.y / 6.0,
                              lq3[2] + ga.z + lv * bc.z / 6.0};
        const double lb[3] = {lq3[0] + gb.x + lv * ca.x / 6.0, lq3[1] + gb.y + lv * ca.y / 6.0,
                              lq3[2] + gb.z + lv * ca.z / 6.0};
        const double lc[3] = {lq3[0] + gc.x + lv * ab.x / 6.0, lq3[1] + gc.y + lv * ab.y / 6.0,
                              lq3[2] + gc.z + lv * ab.z / 6.0};
        for (int k = 0; k < 3; ++k) {
            g[3 * T[0] + k] += la[k];
            g[3 * T[1] + k] += lb[k];
            g[3 * T[2] + k] += lc[k];
            lo[k] -= la[k] + lb[k] + lc[k];
        }
    }
    for (int v = 0; v < nv; ++v)
        for (int k = 0; k < 3; ++k) g[3 * v + k] += lo[k] / nv;
    return J;
}

ibl_status enter(ibl_ctx* ctx) {
    CK(cudaEventRecord(ctx->ev_in, ctx->user_stream));
    CK(cudaStreamWaitEvent(ctx->work, ctx->ev_in, 0));
    return IBL_OK;
}

ibl_status leave(ibl_ctx* ctx) {
    CK(cudaEventRecord(ctx->ev_out, ctx->work));
    CK(cudaStreamWaitEvent(ctx->user_stream, ctx->ev_out, 0));
    return IBL_OK;
}

// Lattice-kernel blocks for the current block size: one warp per group of 32
// fluid nodes.
void layout_tiles(ibl_ctx* ctx) {
    const int per_block = ctx->threads / 32;
    const int blocks = (ctx->dev.n_groups + per_block - 1) / per_block;
    ctx->dev.threads = ctx->threads;
    ctx->dev.lbm_blocks = blocks;
    ctx->dev.lbm_bblocks = (ctx->dev.n_bgroups + per_block - 1) / per_block;
    ctx->dev.grid_lbm = ctx->blocks_per_sm > 0 ? std::min(blocks, ctx->blocks_per_sm * ctx->n_sm) : 0;
    ctx->dev.n_sm = ctx->n_sm;
}

void drop_graphs(ibl_ctx* ctx) {
    for (auto& g : ctx->graph)
        if (g) { cudaGraphExecDestroy(g); g = nullptr; }
    for (auto& g : ctx->adj.graphs) cudaGraphExecDestroy(g.exec);
    ctx->adj.graphs.clear();
}

void free_adjoint(ibl_ctx* ctx) {
    auto& A = ctx->adj;
    for (auto& g : A.graphs) cudaGraphExecDestroy(g.exec);
    A.graphs.clear();
    void* ptrs[] = {A.ck,   A.snap,  A.tape_rhou, A.tape_dvdq, A.tape_rho, A.lamA,   A.lamB,
                    A.acc,  A.tape_F, A.tape_x,  A.tape_v,   A.cp.lx,    A.cp.lxp, A.cp.lv,
                    A.cp.lU, A.cp.lF, A.cp.ln,   A.cp.lA,    A.cp.snorm, A.cp.lV,  A.cp.lfib,
                    A.cp.lmac, A.tape2_rhou, A.tape2_F, A.tape2_dvdq, A.tape2_rho, A.tape2_x, A.tape2_v,
                    A.rx, A.rxm, A.rvacc, A.rnrm, A.rarea, A.rsums};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    for (cudaEvent_t e : {A.ev_rec[0], A.ev_rec[1], A.ev_rev[0], A.ev_rev[1], A.ev_fwd})
        if (e) cudaEventDestroy(e);
    if (A.rs) cudaStreamDestroy(A.rs);
    A = ibl_ctx::AdjCache{};
}

// Owned x-ranges of n slabs, balanced by plane weights (cumulative-weight
// cuts, then pushed apart so that every slab is at least max(H, 1) planes
// wide), and the ghost planes of each side.
bool plan_slabs(int nx, bool per, int S, int H, const double* w, std::vector<ibl_slab>& out, std::string& why) {
    const int wmin = std::max(H, 1);
    if (S < 1 || H < 0 || nx < S * wmin) {
        why = "slab plan: need n_slabs >= 1, halo >= 0 and nx >= n_slabs * max(halo, 1)";
        return false;
    }
    std::vector<double> cum(nx + 1, 0.0);
    for (int x = 0; x < nx; ++x) {
        const double v = w ? w[x] : 1.0;
        if (!(v >= 0.0)) {
            why = "slab plan: negative plane weight";
            return false;
        }
        cum[x + 1] = cum[x] + v;
    }
    if (!(cum[nx] > 0.0))
        for (int x = 0; x <= nx; ++x) cum[x] = x;   // all weights zero: uniform
    std::vector<int> cut(S + 1, 0);
    cut[S] = nx;
    for (int s = 1; s < S; ++s) {
        const double target = cum[nx] * s / S;
        int c = (int)(std::lower_bound(cum.begin(), cum.end(), target) - cum.begin());
        c = std::max(c, cut[s - 1] + wmin);
        c = std::min(c, nx - (S - s) * wmin);
        cut[s] = c;
    }
    out.assign(S, ibl_slab{});
    for (int s = 0; s < S; ++s) {
        ibl_slab& b = out[s];
        b.x0 = cut[s];
        b.x1 = cut[s + 1];
        if (S == 1) { b.lo = b.hi = 0; continue; }
        b.lo = per ? H : std::min(H, b.x0);
        b.hi = per ? H : std::min(H, nx - b.x1);
    }
    return true;
}

// Slab s of the one-lattice member W: its owned planes and ghost planes as a
// lattice of its own (non-periodic in x when cut; a cut face is FACE_HALO),
// with the wall links that start on its planes and end inside them, the face
// data and the initial state of those planes.
bool crop_slab(const MemberHost& W, const ibl_slab& b, int S, MemberHost& M, std::string& why) {
    const auto& d = W.desc;
    const int nx = d.nx, ny = d.ny, nz = d.nz;
    const int nxs = (b.x1 - b.x0) + b.lo + b.hi;
    auto gx_of = [&](int l) { return (((b.x0 - b.lo + l) % nx) + nx) % nx; };
    M = MemberHost{};
    M.desc = d;
    M.desc.nx = nxs;
    if (S > 1) M.desc.periodic[0] = 0;
    const size_t Ns = (size_t)nxs * ny * nz;
    M.tag.assign(Ns, 1);
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int l = 0; l < nxs; ++l)
                M.tag[l + (size_t)nxs * (y + (size_t)ny * z)] = W.tag[gx_of(l) + (size_t)nx * (y + (size_t)ny * z)];
    // links grouped by the global x of their node
    std::vector<std::vector<size_t>> by_x(nx);
    for (size_t i = 0; i < W.links.size(); ++i) by_x[W.links[i].node % (uint32_t)nx].push_back(i);
    for (int l = 0; l < nxs; ++l)
        for (size_t i : by_x[gx_of(l)]) {
            ibl_wall_link L = W.links[i];
            const int tl = l + ex((int)L.dir);
            if (tl < 0 || tl >= nxs) continue;   // leaves the slab: only at its outermost planes
            const uint32_t rest = L.node / (uint32_t)nx;   // y + ny z
            L.node = (uint32_t)l + (uint32_t)nxs * rest;
            M.links.push_back(L);
        }
    for (int f = 0; f < 6; ++f) {
        M.face_kind[f] = W.face_kind[f];
        M.face_rho[f] = W.face_rho[f];
    }
    if (S > 1) {
        if (d.periodic[0] || b.x0 > 0) M.face_kind[0] = FACE_HALO;
        if (d.periodic[0] || b.x1 < nx) M.face_kind[1] = FACE_HALO;
    }
    for (int f = 0; f < 6; ++f) {
        if (W.face_kind[f] != IBL_FACE_VELOCITY || M.face_kind[f] == FACE_HALO) continue;
        const std::vector<float>& v = W.face_vel[f];
        if (f < 2) { M.face_vel[f] = v; continue; }
        // faces 2/3: x + nx z; faces 4/5: x + nx y
        const int other = f < 4 ? nz : ny;
        M.face_vel[f].assign((size_t)3 * nxs * other, 0.f);
        for (int o = 0; o < other; ++o)
            for (int l = 0; l < nxs; ++l)
                for (int c = 0; c < 3; ++c)
                    M.face_vel[f][3 * (l + (size_t)nxs * o) + c] = v[3 * (gx_of(l) + (size_t)nx * o) + c];
    }
    if (!W.init_rho.empty() || !W.init_u.empty()) {
        if (!W.init_rho.empty()) M.init_rho.assign(Ns, 1.f);
        if (!W.init_u.empty()) M.init_u.assign(3 * Ns, 0.f);
        for (int z = 0; z < nz; ++z)
            for (int y = 0; y < ny; ++y)
                for (int l = 0; l < nxs; ++l) {
                    const size_t ln = l + (size_t)nxs * (y + (size_t)ny * z);
                    const size_t gn = gx_of(l) + (size_t)nx * (y + (size_t)ny * z);
                    if (!W.init_rho.empty()) M.init_rho[ln] = W.init_rho[gn];
                    if (!W.init_u.empty())
                        for (int c = 0; c < 3; ++c) M.init_u[3 * ln + c] = W.init_u[3 * gn + c];
                }
    }
    return true;
}

ibl_status validate_member(ibl_ctx* ctx, const MemberHost& M) {
    const auto& d = M.desc;
    const long long N = (long long)d.nx * d.ny * d.nz;
    if ((long long)M.tag.size() != N) return fail(ctx, IBL_ERR_STATE, "geometry not set");
    const int dims[3] = {d.nx, d.ny, d.nz};
    // only nodes on a non-periodic box face can break the rule: every row
    // (fixed y, z) on a y or z face is scanned whole, every other row at its
    // two x ends, in node order (the first bad node is the one reported)
    auto check = [&](int x, int y, int z) -> ibl_status {
        const long long n = x + (long long)d.nx * (y + (long long)d.ny * z);
        if (M.tag[n] != 0) return IBL_OK;
        const int c[3] = {x, y, z};
        int nf = 0, face = -1;
        for (int a = 0; a < 3; ++a) {
            if (d.periodic[a]) continue;
            if (c[a] == 0 && M.face_kind[2 * a] != FACE_HALO) { ++nf; face = 2 * a; }
            if (c[a] == dims[a] - 1 && M.face_kind[2 * a + 1] != FACE_HALO) { ++nf; face = 2 * a + 1; }
        }
        if (nf > 1)
            return fail(ctx, IBL_ERR_ARG, "fluid node " + std::to_string(n) + " lies on an edge of the box (two faces)");
        if (nf == 1 && M.face_kind[face] == IBL_FACE_NONE)
            return fail(ctx, IBL_ERR_ARG, "fluid node " + std::to_string(n) + " lies on face " + std::to_string(face) +
                                              " which has no velocity or pressure condition");
        return IBL_OK;
    };
    for (int z = 0; z < d.nz; ++z)
        for (int y = 0; y < d.ny; ++y) {
            const bool row_on_face = (!d.periodic[1] && (y == 0 || y == d.ny - 1)) ||
                                     (!d.periodic[2] && (z == 0 || z == d.nz - 1));
            if (row_on_face) {
                for (int x = 0; x < d.nx; ++x) CKS(check(x, y, z));
            } else if (!d.periodic[0]) {
                CKS(check(0, y, z));
                if (d.nx > 1) CKS(check(d.nx - 1, y, z));
            }
        }
    return IBL_OK;
}

// ---------------------------------------------------------------------------
// Static staging array of ibl_read_fields_noalloc, for callers that may not
// allocate device memory: rho in the first IBL_NOALLOC_MAX_NODES floats, u in
// the next 3 * IBL_NOALLOC_MAX_NODES.  Nothing in it needs to start at zero:
// the read kernel writes every element that is then copied out (solid nodes
// as 0).  One array per device, shared by every context of the process, so
// overlapping calls race on it.  Its device address is looked up while a
// context is set up (finalize), which allocates anyway: that lookup loads
// this file's module, and with it the array, under lazy module loading, so
// the entry point itself neither loads a module nor reserves memory.
// ---------------------------------------------------------------------------
}  // namespace

static __device__ __align__(256) float g_noalloc_scratch[4 * (size_t)IBL_NOALLOC_MAX_NODES];

namespace {

constexpr int NOALLOC_MAX_DEVICES = 64;
std::mutex g_noalloc_mu;
float* g_noalloc_ptr[NOALLOC_MAX_DEVICES] = {};

// Address of device dev's copy of the static array (dev must be the current
// device), looked up once per device and cached.
ibl_status noalloc_scratch(ibl_ctx* ctx, int dev, float** out) {
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return fail(ctx, IBL_ERR_ARG, "device ordinal beyond 63");
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return fail(ctx, IBL_ERR_CUDA, std::string("cudaGetSymbolAddress of the static read array failed: ") +
                                               cudaGetErrorString(e));
        g_noalloc_ptr[dev] = (float*)p;
    }
    *out = g_noalloc_ptr[dev];
    return IBL_OK;
}

// Chunks of the staged lattice kernel (a context of one lattice): every run
// of consecutive interior fluid nodes of the work list cut into pieces of at
// most lbm_chunk_nodes() nodes.  Built when that kernel is first asked for.
ibl_status build_chunks(ibl_ctx* ctx, const std::vector<uint32_t>& nodes) {
    DevState& D = ctx->dev;
    if (ctx->members.size() != 1 || D.n_groups == 0 || D.chunks) return IBL_OK;
    std::vector<uint2> ch;
    const uint32_t cap = (uint32_t)lbm_chunk_nodes();
    for (size_t i = 0; i < nodes.size() && nodes[i] != NO_NODE; ++i) {
        const uint32_t n = nodes[i];
        if (ch.empty() || n != ch.back().x + ch.back().y || ch.back().y == cap) ch.push_back(make_uint2(n, 1u));
        else ch.back().y += 1;
    }
    D.n_chunks = (int)ch.size();
    CKS(dev_alloc(ctx, D.chunks, ch.size()));
    CKS(upload(ctx, D.chunks, ch));
    return IBL_OK;
}

// the staged kernel's shared-memory attribute and residency (0 blocks: the
// layout does not allow it and the register kernel runs)
ibl_status prepare_staged(ibl_ctx* ctx) {
    DevState& D = ctx->dev;
    D.bulk_blocks_per_sm = 0;
    if (D.chunks && lbm_bulk_layout_ok(D)) {
        int nb = 0;
        CK(lbm_bulk_prepare(D.storage, nb));
        D.bulk_blocks_per_sm = nb;
    }
    return IBL_OK;
}

ibl_status finalize(ibl_ctx* ctx) {
    if (ctx->finalized) return IBL_OK;
    int dev_id = 0;
    CK(cudaGetDevice(&dev_id));
    if (dev_id != ctx->device)
        return fail(ctx, IBL_ERR_STATE, "the context's device (" + std::to_string(ctx->device) +
                                            ") must be current when it is set up");
    CK(cudaDeviceGetAttribute(&ctx->n_sm, cudaDevAttrMultiProcessorCount, dev_id));
    // the static array of ibl_read_fields_noalloc: looked up here, where the
    // set-up allocates anyway, so that the entry point itself loads nothing
    CKS(noalloc_scratch(ctx, dev_id, &ctx->noalloc));
    const int nm = (int)ctx->members.size();
    if (nm < 1 || nm > MAX_MEMBERS) return fail(ctx, IBL_ERR_ARG, "member count out of range");
    for (auto& M : ctx->members)
        if (!M.whole_view) CKS(validate_member(ctx, M));

    const size_t esize = ctx->storage == IBL_STORAGE_F32 ? 4 : 2;
    DevState& D = ctx->dev;
    D.storage = ctx->storage;
    D.n_members = nm;
    ctx->hmem.assign(nm, MemberDev{});
    long long f_off = 0, node_off = 0, face_off = 0, cell_off = 0;
    int link_off = 0, cap_off = 0, vert_off = 0;
    std::vector<uint8_t> tag_all;
    std::vector<float> face_all;
    std::vector<uint32_t> l_node, l_meta;
    std::vector<float> l_q, l_dq;
    // capsule arrays
    std::vector<CapsuleDev> caps;
    std::vector<int> v_cap, tri_all, hinge_all, e_cap;
    std::vector<double> x_all, vel_all;
    std::vector<float> l0_all, ks_all, th0_all, kb_all;
    int max_nv = 0, tri_off = 0, edge_off = 0;
    bool any_soft = false, any_rigid = false, any_cells = false;
    ctx->member_caps.assign(nm, {});

    for (int mi = 0; mi < nm; ++mi) {
        const MemberHost& M = ctx->members[mi];
        const auto& d = M.desc;
        MemberDev& md = ctx->hmem[mi];
        md.nx = d.nx; md.ny = d.ny; md.nz = d.nz;
        md.px = d.periodic[0] ? 0 : 1; md.py = d.periodic[1] ? 0 : 1; md.pz = d.periodic[2] ? 0 : 1;
        md.per = (d.periodic[0] ? 1 : 0) | (d.periodic[1] ? 2 : 0) | (d.periodic[2] ? 4 : 0);
        md.NX = d.nx + 2 * md.px; md.NY = d.ny + 2 * md.py; md.NZ = d.nz + 2 * md.pz;
        const long long Np = (long long)md.NX * md.NY * md.NZ;
        if (Np * 19 >= (1LL << 31)) return fail(ctx, IBL_ERR_ARG, "lattice too large for one member");
        md.N = (int)Np;
        md.S = (int)round_up((size_t)Np, 64) + IBL_PLANE_PAD;
        md.f_off = M.whole_view ? 0 : f_off;
        md.node_off = node_off;
        md.slab_view = M.whole_view ? 1 : 0;
        if (!M.whole_view) f_off += 19LL * md.S;
        node_off += (long long)round_up((size_t)Np, 256);
        md.omega = (float)(1.0 / d.tau);
        md.guo = (float)(1.0 - 0.5 / d.tau);
        md.nu = (float)((d.tau - 0.5) / 3.0);
        md.umax = (float)d.u_max;
        for (int a = 0; a < 3; ++a) md.F[a] = (float)d.body_force[a];
        md.hasF = (d.body_force[0] != 0 || d.body_force[1] != 0 || d.body_force[2] != 0) ? 1 : 0;
        md.st_scale = ctx->storage == IBL_STORAGE_F16 ? 4096.f : 1.f;
        md.ld_scale = ctx->storage == IBL_STORAGE_F16 ? 1.f / 4096.f : 1.f;
        for (int fc = 0; fc < 6; ++fc) {
            md.face_kind[fc] = M.face_kind[fc];
            md.face_rho[fc] = (float)M.face_rho[fc];
            md.face_off[fc] = -1;
            if (M.face_kind[fc] == IBL_FACE_VELOCITY) {
                md.face_off[fc] = face_off;
                face_all.insert(face_all.end(), M.face_vel[fc].begin(), M.face_vel[fc].end());
                face_off += (long long)M.face_vel[fc].size() / 3;
            }
        }
        // padded tags (ghost layer solid)
        const size_t base = tag_all.size();
        tag_all.resize(base + round_up((size_t)Np, 256), TAG_SOLID);
        parallel_chunks((size_t)d.nz, 4, [&](size_t z0, size_t z1) {
            for (int z = (int)z0; z < (int)z1; ++z)
                for (int y = 0; y < d.ny; ++y)
                    for (int x = 0; x < d.nx; ++x) {
                        const long long un = x + (long long)d.nx * (y + (long long)d.ny * z);
                        const long long pn =
                            (x + md.px) + (long long)md.NX * ((y + md.py) + (long long)md.NY * (z + md.pz));
                        tag_all[base + pn] = M.tag[un] ? TAG_SOLID : 0;
                    }
        });
        // links
        md.link_begin = link_off;
        const int dims[3] = {d.nx, d.ny, d.nz};
        auto shift = [&](int c[3], int s, int k, int out[3]) -> bool {
            const int e[3] = {ex(k), ey(k), ez(k)};
            bool ok = true;
            for (int a = 0; a < 3; ++a) {
                int v = c[a] + s * e[a];
                if (d.periodic[a]) v = ((v % dims[a]) + dims[a]) % dims[a];
                else if (v < 0 || v >= dims[a]) ok = false;
                out[a] = v;
            }
            return ok;
        };
        auto fluid_at = [&](int c[3]) { return M.tag[c[0] + (long long)d.nx * (c[1] + (long long)d.ny * c[2])] == 0; };
        // the member's links in (direction, node) order: consecutive threads
        // of the wall pass then touch consecutive nodes of one population
        // plane along a wall
        struct LinkRec { uint32_t node, meta; float q, dq; };
        const size_t nl = M.links.size();
        std::vector<LinkRec> made(nl);
        // per link: 0 valid, 1 out of range, 2 starts at a solid node, 3 does
        // not end at a solid node inside the box; the first bad link is reported
        std::vector<uint8_t> bad(nl, 0);
        parallel_chunks(nl, 16384, [&](size_t l0, size_t l1) {
            const long long Nu = (long long)d.nx * d.ny * d.nz;
            for (size_t li = l0; li < l1; ++li) {
                const ibl_wall_link& L = M.links[li];
                if ((long long)L.node >= Nu || L.dir < 1 || L.dir > 18 || !(L.q > 0.f && L.q <= 1.f)) { bad[li] = 1; continue; }
                int c[3] = {(int)(L.node % d.nx), (int)((L.node / d.nx) % d.ny), (int)(L.node / ((long long)d.nx * d.ny))};
                int s0[3], m1[3], m2[3];
                if (!fluid_at(c)) { bad[li] = 2; continue; }
                if (!shift(c, 1, L.dir, s0) || fluid_at(s0)) { bad[li] = 3; continue; }
                const bool ok1 = shift(c, -1, L.dir, m1) && fluid_at(m1);
                const bool ok2 = shift(c, -2, L.dir, m2) && fluid_at(m2);
                const long long pn =
                    (c[0] + md.px) + (long long)md.NX * ((c[1] + md.py) + (long long)md.NY * (c[2] + md.pz));
                made[li] = {(uint32_t)pn, L.dir | (ok1 ? 32u : 0u) | (ok2 ? 64u : 0u) | ((uint32_t)mi << 8), L.q, L.dq};
            }
        });
        for (size_t li = 0; li < nl; ++li)
            if (bad[li])
                return fail(ctx, IBL_ERR_ARG, "wall link " + std::to_string(li) +
                                                  (bad[li] == 1 ? " out of range"
                                                   : bad[li] == 2 ? " starts at a solid node"
                                                                  : " does not end at a solid node inside the box"));
        // (direction, node) order: a stable counting sort by direction over
        // fixed pieces of the list (per-piece counts, then each piece scattered
        // by a host thread to its offsets in the member's part of the link
        // arrays), then each direction's run sorted by node unless it already is
        {
            const size_t P = std::max<size_t>(1, std::min<size_t>(64, nl / 65536));
            const size_t step = (nl + P - 1) / P;
            std::vector<size_t> cnt(P * 20, 0);
            parallel_chunks(P, 1, [&](size_t p0, size_t p1) {
                for (size_t pi = p0; pi < p1; ++pi)
                    for (size_t li = pi * step; li < std::min(nl, (pi + 1) * step); ++li)
                        ++cnt[pi * 20 + (made[li].meta & 31u)];
            });
            // start of every (direction, piece) block: directions outer, pieces inner
            std::vector<size_t> at(P * 20, 0), dir_begin(20, 0);
            size_t run = 0;
            for (int k = 0; k < 20; ++k) {
                dir_begin[k] = run;
                for (size_t pi = 0; pi < P; ++pi) {
                    at[pi * 20 + k] = run;
                    run += cnt[pi * 20 + k];
                }
            }
            const size_t o = l_node.size();
            l_node.resize(o + nl);
            l_meta.resize(o + nl);
            l_q.resize(o + nl);
            l_dq.resize(o + nl);
            parallel_chunks(P, 1, [&](size_t p0, size_t p1) {
                for (size_t pi = p0; pi < p1; ++pi) {
                    size_t* pos = &at[pi * 20];
                    for (size_t li = pi * step; li < std::min(nl, (pi + 1) * step); ++li) {
                        const LinkRec& r = made[li];
                        const size_t j = o + pos[r.meta & 31u]++;
                        l_node[j] = r.node;
                        l_meta[j] = r.meta;
                        l_q[j] = r.q;
                        l_dq[j] = r.dq;
                    }
                }
            });
            parallel_chunks(19, 1, [&](size_t k0, size_t k1) {
                for (size_t k = std::max<size_t>(k0, 1); k < k1; ++k) {
                    const size_t b = o + dir_begin[k], e = o + dir_begin[k + 1];
                    bool sorted = true;
                    for (size_t j = b + 1; j < e && sorted; ++j) sorted = l_node[j - 1] <= l_node[j];
                    if (sorted) continue;
                    std::vector<size_t> idx(e - b);
                    for (size_t j = 0; j < idx.size(); ++j) idx[j] = b + j;
                    std::stable_sort(idx.begin(), idx.end(), [&](size_t x, size_t y) { return l_node[x] < l_node[y]; });
                    std::vector<uint32_t> nn(idx.size()), mm(idx.size());
                    std::vector<float> qq(idx.size()), dd(idx.size());
                    for (size_t j = 0; j < idx.size(); ++j) {
                        nn[j] = l_node[idx[j]]; mm[j] = l_meta[idx[j]]; qq[j] = l_q[idx[j]]; dd[j] = l_dq[idx[j]];
                    }
                    std::copy(nn.begin(), nn.end(), l_node.begin() + b);
                    std::copy(mm.begin(), mm.end(), l_meta.begin() + b);
                    std::copy(qq.begin(), qq.end(), l_q.begin() + b);
                    std::copy(dd.begin(), dd.end(), l_dq.begin() + b);
                }
            });
        }
        md.link_count = (int)M.links.size();
        link_off += md.link_count;
        // capsules
        md.cap_begin = cap_off;
        md.cap_count = (int)M.caps.size();
        md.vert_begin = vert_off;
        const double nu = (d.tau - 0.5) / 3.0;
        // per capsule, on host threads: hinges, FP64 sums, rest lengths,
        // spring and bending constants and rest angles
        struct CapPre {
            std::vector<int> hinge, ta, tb;
            MeshSums ms;
            double radius = 0.0;
            std::vector<double> l0;
            std::vector<float> ks, kb, th0;
            std::string why;
        };
        std::vector<CapPre> pre(M.caps.size());
        parallel_chunks(M.caps.size(), 1, [&](size_t c0, size_t c1) {
            for (size_t ci = c0; ci < c1; ++ci) {
                const CapsuleHost& ch = M.caps[ci];
                CapPre& P = pre[ci];
                const int nv = (int)ch.X.size() / 3, nt = (int)ch.tris.size() / 3;
                if (!build_hinges(ch.tris, nv, P.hinge, P.ta, P.tb, P.why)) {
                    P.why = "capsule " + std::to_string(ci) + " mesh: " + P.why;
                    continue;
                }
                const double* X = ch.X.data();
                P.ms = mesh_sums(X, nv, ch.tris.data(), nt);
                if (!(P.ms.V > 0)) {
                    P.why = "capsule " + std::to_string(ci) + " mesh encloses no volume (triangles must be outward CCW)";
                    continue;
                }
                std::vector<double> tri_area(nt);
                for (int t = 0; t < nt; ++t) {
                    const int* T = &ch.tris[3 * t];
                    const V3 a = {X[3 * T[0]], X[3 * T[0] + 1], X[3 * T[0] + 2]};
                    const V3 b = {X[3 * T[1]], X[3 * T[1] + 1], X[3 * T[1] + 2]};
                    const V3 c = {X[3 * T[2]], X[3 * T[2] + 1], X[3 * T[2] + 2]};
                    tri_area[t] = 0.5 * vnorm(vcross(vsub(b, a), vsub(c, a)));
                }
                P.radius = std::cbrt(3.0 * P.ms.V / (4.0 * M_PI));
                const double ks0 = ch.p.Ca > 0 ? nu * ch.p.u_ref / ch.p.Ca : 0.0;   // Ca = rho nu u_ref / k_s0
                const int ne = (int)P.hinge.size() / 4;
                P.l0.resize(ne);
                P.ks.resize(ne);
                P.kb.resize(ne);
                P.th0.resize(ne);
                for (int e = 0; e < ne; ++e) {
                    const int* h = &P.hinge[4 * e];
                    const V3 p1 = {X[3 * h[0]], X[3 * h[0] + 1], X[3 * h[0] + 2]};
                    const V3 p2 = {X[3 * h[1]], X[3 * h[1] + 1], X[3 * h[1] + 2]};
                    const V3 p3 = {X[3 * h[2]], X[3 * h[2] + 1], X[3 * h[2] + 2]};
                    const V3 p4 = {X[3 * h[3]], X[3 * h[3] + 1], X[3 * h[3] + 2]};
                    const double l0 = vnorm(vsub(p3, p2));
                    const double ks = ks0 * (tri_area[P.ta[e]] + tri_area[P.tb[e]]) / (l0 * l0);   // T = 1
                    const double kb = ch.p.Eb * ks * P.radius * P.radius;                         // Eb = k_b/(k_s,l r^2)
                    P.l0[e] = l0;
                    P.ks[e] = (float)ks;
                    P.kb[e] = (float)kb;
                    P.th0[e] = (float)signed_dihedral(p1, p2, p3, p4);
                }
            }
        });
        for (size_t ci = 0; ci < M.caps.size(); ++ci) {
            const CapsuleHost& ch = M.caps[ci];
            const CapPre& P = pre[ci];
            if (!P.why.empty()) return fail(ctx, IBL_ERR_ARG, P.why);
            const int nv = (int)ch.X.size() / 3, nt = (int)ch.tris.size() / 3;
            const int ne = (int)P.hinge.size() / 4;
            const double* X = ch.X.data();
            const MeshSums& ms = P.ms;
            const double radius = P.radius;
            CapsuleDev cd{};
            cd.member = mi;
            cd.rigid = ch.p.rigid ? 1 : 0;
            cd.v_begin = vert_off; cd.v_count = nv;
            cd.t_begin = tri_off; cd.t_count = nt;
            cd.e_begin = edge_off; cd.e_count = ne;
            cd.kv = ch.p.kv; cd.V0 = ms.V; cd.inv_V0 = 1.0 / ms.V; cd.S0 = ms.S;
            cd.mass = ch.p.density_ratio * ms.V;
            cd.mv = cd.mass / nv;
            cd.inertia = 0.4 * cd.mass * radius * radius;
            cd.xc[0] = ms.cen.x; cd.xc[1] = ms.cen.y; cd.xc[2] = ms.cen.z;
            for (int a = 0; a < 3; ++a) { cd.u1[a] = cd.u2[a] = ch.vel0[a]; cd.w1[a] = cd.w2[a] = 0.0; }
            CapsuleRestHost rh;
            rh.member = mi; rh.v_begin = vert_off; rh.nv = nv; rh.t_begin = tri_off; rh.nt = nt;
            rh.e_begin = edge_off; rh.ne = ne; rh.S0 = ms.S; rh.V0 = ms.V; rh.rigid = cd.rigid;
            rh.l0 = P.l0;
            rh.edges.reserve(2 * (size_t)ne);
            for (int e = 0; e < ne; ++e) {
                const int* h = &P.hinge[4 * e];
                for (int j = 0; j < 4; ++j) hinge_all.push_back(vert_off + h[j]);
                l0_all.push_back((float)P.l0[e]);
                e_cap.push_back(cap_off);
                rh.edges.push_back(h[1]);
                rh.edges.push_back(h[2]);
            }
            ks_all.insert(ks_all.end(), P.ks.begin(), P.ks.end());
            kb_all.insert(kb_all.end(), P.kb.begin(), P.kb.end());
            th0_all.insert(th0_all.end(), P.th0.begin(), P.th0.end());
            for (int t = 0; t < nt; ++t)
                for (int j = 0; j < 3; ++j) tri_all.push_back(vert_off + ch.tris[3 * t + j]);
            for (int v = 0; v < nv; ++v) {
                v_cap.push_back(cap_off);
                for (int a = 0; a < 3; ++a) {
                    x_all.push_back(X[3 * v + a]);
                    vel_all.push_back(ch.vel0[a]);
                }
            }
            caps.push_back(cd);
            ctx->rest.push_back(rh);
            ctx->member_caps[mi].push_back(cap_off);
            max_nv = std::max(max_nv, nv);
            any_soft |= !cd.rigid;
            any_rigid |= (bool)cd.rigid;
            ++cap_off;
            vert_off += nv;
            tri_off += nt;
            edge_off += ne;
        }
        md.vert_count = vert_off - md.vert_begin;
        md.has_cells = md.cap_count >= 2 ? 1 : 0;
        md.cell_off = cell_off;
        md.cnx = (d.nx + 1) / 2; md.cny = (d.ny + 1) / 2; md.cnz = (d.nz + 1) / 2;
        if (md.has_cells) {
            cell_off += (long long)md.cnx * md.cny * md.cnz;
            any_cells = true;
        }
    }
    if (max_nv > 12000) return fail(ctx, IBL_ERR_ARG, "a capsule has more than 12000 vertices");

    // fluid-segment work lists of the lattice kernel: aligned 32-node runs of
    // the padded layout holding at least one fluid node, split into border
    // runs (a fluid node on the wrap plane of a periodic axis: coordinates
    // needed) and interior runs; and the list of fluid nodes on Zou-He faces
    std::vector<uint32_t> segs, bsegs, fc_node, fc_meta, nodes, bnodes;
    std::vector<int> group_mem, bgroup_mem;
    {
        size_t base = 0;
        for (int m = 0; m < nm; ++m) {
            MemberDev& md = ctx->hmem[m];
            md.seg_begin = (int)segs.size();
            md.bseg_begin = (int)bsegs.size();
            if (ctx->members[m].whole_view) {   // no lattice work
                md.seg_count = md.bseg_count = 0;
                base += round_up((size_t)md.N, 256);
                continue;
            }
            const int ns = (md.N + 31) / 32;
            const bool per[3] = {(md.per & 1) != 0, (md.per & 2) != 0, (md.per & 4) != 0};
            const int dimP[3] = {md.NX, md.NY, md.NZ};
            // runs of segments scanned on host threads into lists of their
            // own, joined in segment order (the same lists as one scan)
            struct Part { std::vector<uint32_t> segs, bsegs, nodes, bnodes, fc_node, fc_meta; };
            const size_t n_parts = std::min<size_t>(64, std::max<size_t>(1, (size_t)ns / 2048));
            std::vector<Part> part(n_parts);
            const size_t per_part = ((size_t)ns + n_parts - 1) / n_parts;
            parallel_chunks(n_parts, 1, [&](size_t p0, size_t p1) {
                for (size_t pi = p0; pi < p1; ++pi) {
                    Part& P = part[pi];
                    const int j0 = (int)std::min((size_t)ns, pi * per_part);
                    const int j1 = (int)std::min((size_t)ns, (pi + 1) * per_part);
                    const long long n0 = 32LL * j0;
                    // coordinates of node n, kept by counters (no divisions)
                    int c[3] = {(int)(n0 % md.NX), (int)((n0 / md.NX) % md.NY), (int)(n0 / ((long long)md.NX * md.NY))};
                    for (int j = j0; j < j1; ++j) {
                        bool any = false, border = false;
                        for (int t = 0; t < 32; ++t) {
                            const long long n = 32LL * j + t;
                            if (n >= md.N) break;
                            if (!(tag_all[base + n] & TAG_SOLID)) {
                                any = true;
                                int face = -1;
                                bool wrap = false;
                                for (int a = 0; a < 3; ++a) {
                                    if (per[a] && (c[a] == 0 || c[a] == dimP[a] - 1)) wrap = true;    // wrap plane
                                    if (!per[a] && face < 0 && c[a] == 1 && md.face_kind[2 * a] != FACE_HALO)
                                        face = 2 * a;                                                  // box faces
                                    if (!per[a] && face < 0 && c[a] == dimP[a] - 2 &&
                                        md.face_kind[2 * a + 1] != FACE_HALO)
                                        face = 2 * a + 1;
                                }
                                border = border || wrap;
                                (wrap ? P.bnodes : P.nodes).push_back((uint32_t)n);
                                if (face >= 0 &&
                                    (md.face_kind[face] == FACE_VELOCITY || md.face_kind[face] == FACE_PRESSURE)) {
                                    P.fc_node.push_back((uint32_t)n);
                                    P.fc_meta.push_back((uint32_t)face | ((uint32_t)m << 8));
                                }
                            }
                            if (++c[0] == md.NX) { c[0] = 0; if (++c[1] == md.NY) { c[1] = 0; ++c[2]; } }
                        }
                        if (any) (border ? P.bsegs : P.segs).push_back((uint32_t)j);
                    }
                }
            });
            for (const Part& P : part) {
                segs.insert(segs.end(), P.segs.begin(), P.segs.end());
                bsegs.insert(bsegs.end(), P.bsegs.begin(), P.bsegs.end());
                nodes.insert(nodes.end(), P.nodes.begin(), P.nodes.end());
                bnodes.insert(bnodes.end(), P.bnodes.begin(), P.bnodes.end());
                fc_node.insert(fc_node.end(), P.fc_node.begin(), P.fc_node.end());
                fc_meta.insert(fc_meta.end(), P.fc_meta.begin(), P.fc_meta.end());
            }
            // close the member's node lists on a whole group of 32
            for (auto* lst : {&nodes, &bnodes}) {
                while (lst->size() % 32) lst->push_back(NO_NODE);
                std::vector<int>& gm = lst == &nodes ? group_mem : bgroup_mem;
                gm.resize(lst->size() / 32, m);
            }
            md.seg_count = (int)segs.size() - md.seg_begin;
            md.bseg_count = (int)bsegs.size() - md.bseg_begin;
            base += round_up((size_t)md.N, 256);
        }
        D.n_segs = (int)segs.size();
        D.n_bsegs = (int)bsegs.size();
        D.n_groups = (int)(nodes.size() / 32);
        D.n_bgroups = (int)(bnodes.size() / 32);
        D.n_face_nodes = (int)fc_node.size();
    }
    layout_tiles(ctx);
    // device buffers
    CKS(dev_alloc(ctx, D.segs, std::max<size_t>(segs.size(), 1)));
    CKS(dev_alloc(ctx, D.bsegs, std::max<size_t>(bsegs.size(), 1)));
    CKS(upload(ctx, D.segs, segs));
    CKS(upload(ctx, D.bsegs, bsegs));
    CKS(dev_alloc(ctx, D.nodes, std::max<size_t>(nodes.size(), 1)));
    CKS(dev_alloc(ctx, D.bnodes, std::max<size_t>(bnodes.size(), 1)));
    CKS(upload(ctx, D.nodes, nodes));
    CKS(upload(ctx, D.bnodes, bnodes));
    // the staged lattice kernel's chunks, when that kernel is asked for
    if (ctx->lattice_path == 1) CKS(build_chunks(ctx, nodes));
    if (nm > 1) {
        CKS(dev_alloc(ctx, D.group_mem, std::max<size_t>(group_mem.size(), 1)));
        CKS(dev_alloc(ctx, D.bgroup_mem, std::max<size_t>(bgroup_mem.size(), 1)));
        CKS(upload(ctx, D.group_mem, group_mem));
        CKS(upload(ctx, D.bgroup_mem, bgroup_mem));
    }
    // the wall links that start on a Zou-He face node: taken by that node's
    // thread of the walls kernel, before its face rule
    {
        // face nodes of each member: a bit per padded node (the members'
        // node ranges are disjoint in node_off), then the face node's index by
        // binary search in its member's ascending part of the face list
        std::vector<uint64_t> is_face(((size_t)node_off + 63) / 64, 0);
        std::vector<size_t> fc_begin(nm + 1, fc_node.size());
        for (size_t i = fc_node.size(); i-- > 0;) fc_begin[fc_meta[i] >> 8] = i;
        for (int m = nm - 1; m >= 0; --m) fc_begin[m] = std::min(fc_begin[m], fc_begin[m + 1]);
        for (size_t i = 0; i < fc_node.size(); ++i) {
            const size_t g = (size_t)ctx->hmem[fc_meta[i] >> 8].node_off + fc_node[i];
            is_face[g >> 6] |= 1ull << (g & 63);
        }
        std::vector<std::vector<int>> per(fc_node.size());
        for (size_t l = 0; l < l_node.size(); ++l) {
            const int m = (int)(l_meta[l] >> 8);
            const size_t g = (size_t)ctx->hmem[m].node_off + l_node[l];
            if (!((is_face[g >> 6] >> (g & 63)) & 1ull)) continue;
            const auto b = fc_node.begin() + fc_begin[m], e = fc_node.begin() + fc_begin[m + 1];
            const auto it = std::lower_bound(b, e, l_node[l]);
            per[it - fc_node.begin()].push_back((int)l);
            l_meta[l] |= LINK_AT_FACE;
        }
        std::vector<int> lbeg(fc_node.size() + 1, 0), links;
        for (size_t i = 0; i < per.size(); ++i) {
            lbeg[i + 1] = lbeg[i] + (int)per[i].size();
            links.insert(links.end(), per[i].begin(), per[i].end());
        }
        CKS(dev_alloc(ctx, D.fc_lbeg, lbeg.size()));
        CKS(dev_alloc(ctx, D.fc_links, std::max<size_t>(links.size(), 1)));
        CKS(upload(ctx, D.fc_lbeg, lbeg));
        CKS(upload(ctx, D.fc_links, links));
    }
    CKS(dev_alloc(ctx, D.fc_node, std::max<size_t>(fc_node.size(), 1)));
    CKS(dev_alloc(ctx, D.fc_meta, std::max<size_t>(fc_meta.size(), 1)));
    CKS(upload(ctx, D.fc_node, fc_node));
    CKS(upload(ctx, D.fc_meta, fc_meta));
    D.f_bytes = (size_t)f_off * esize;
    CKS(dev_alloc(ctx, (uint8_t*&)D.f, D.f_bytes));
    CKS(dev_alloc(ctx, D.tag, tag_all.size()));
    CKS(dev_alloc(ctx, D.face_vel, std::max<size_t>(face_all.size(), 3)));
    CKS(dev_alloc(ctx, D.status, nm));
    CKS(dev_alloc(ctx, D.status_new, nm));
    CKS(dev_alloc(ctx, D.counters, nm));
    D.n_links = link_off;
    CKS(dev_alloc(ctx, D.l_node, l_node.size()));
    CKS(dev_alloc(ctx, D.l_meta, l_meta.size()));
    CKS(dev_alloc(ctx, D.l_q, l_q.size()));
    CKS(dev_alloc(ctx, D.l_dq, l_dq.size()));
    CKS(upload(ctx, D.tag, tag_all));
    CKS(upload(ctx, D.face_vel, face_all));
    CKS(upload(ctx, D.l_node, l_node));
    CKS(upload(ctx, D.l_meta, l_meta));
    CKS(upload(ctx, D.l_q, l_q));
    CKS(upload(ctx, D.l_dq, l_dq));
    CK(cudaMemsetAsync(D.status, 0, sizeof(uint32_t) * nm, ctx->work));
    CK(cudaMemsetAsync(D.status_new, 0, sizeof(uint32_t) * nm, ctx->work));
    CK(cudaMemsetAsync(D.counters, 0, sizeof(int) * nm, ctx->work));
    D.n_caps = cap_off; D.n_verts = vert_off; D.n_tris = tri_off; D.n_edges = edge_off;
    D.any_soft = any_soft; D.any_rigid = any_rigid; D.any_cells = any_cells; D.max_nv = max_nv;
    if (cap_off > 0) {
        CKS(dev_alloc(ctx, D.fib, 4 * (size_t)node_off));
        CK(cudaMemsetAsync(D.fib, 0, sizeof(float) * 4 * (size_t)node_off, ctx->work));
        CKS(dev_alloc(ctx, D.caps, caps.size()));
        CKS(dev_alloc(ctx, D.sums, caps.size()));
        CKS(dev_alloc(ctx, D.v_cap, v_cap.size()));
        CKS(dev_alloc(ctx, D.x, x_all.size()));
        CKS(dev_alloc(ctx, D.x_prev, x_all.size()));
        CKS(dev_alloc(ctx, D.xm, 2 * (x_all.size() / 3)));
        CKS(dev_alloc(ctx, D.vel, vel_all.size()));
        CKS(dev_alloc(ctx, D.force, 4 * (x_all.size() / 3)));
        CKS(dev_alloc(ctx, D.uv0, x_all.size()));
        CKS(dev_alloc(ctx, D.nrm, x_all.size()));
        CKS(dev_alloc(ctx, D.area, (size_t)vert_off));
        CKS(dev_alloc(ctx, D.macro, (size_t)node_off));
        CKS(dev_alloc(ctx, D.probe, 16 * (size_t)vert_off));
        CKS(dev_alloc(ctx, D.vacc, (size_t)vert_off));
        CK(cudaMemsetAsync(D.vacc, 0, sizeof(float4) * (size_t)vert_off, ctx->work));
        CK(cudaMemsetAsync(D.probe, 0, sizeof(float) * 16 * (size_t)vert_off, ctx->work));
        CKS(dev_alloc(ctx, D.tri, tri_all.size()));
        CKS(dev_alloc(ctx, D.hinge, hinge_all.size()));
        CKS(dev_alloc(ctx, D.l0, l0_all.size()));
        CKS(dev_alloc(ctx, D.ks, ks_all.size()));
        CKS(dev_alloc(ctx, D.th0, th0_all.size()));
        CKS(dev_alloc(ctx, D.kb, kb_all.size()));
        CKS(dev_alloc(ctx, D.e_cap, e_cap.size()));
        CKS(upload(ctx, D.caps, caps));
        CK(cudaMemsetAsync(D.sums, 0, sizeof(CapsuleSums) * caps.size(), ctx->work));
        CKS(upload(ctx, D.v_cap, v_cap));
        CKS(upload(ctx, D.x, x_all));
        CKS(upload(ctx, D.x_prev, x_all));
        CKS(upload(ctx, D.vel, vel_all));
        CK(cudaMemsetAsync(D.force, 0, sizeof(float) * 4 * (x_all.size() / 3), ctx->work));
        CK(cudaMemsetAsync(D.uv0, 0, sizeof(float) * x_all.size(), ctx->work));
        CKS(upload(ctx, D.tri, tri_all));
        CKS(upload(ctx, D.hinge, hinge_all));
        CKS(upload(ctx, D.l0, l0_all));
        CKS(upload(ctx, D.ks, ks_all));
        CKS(upload(ctx, D.th0, th0_all));
        CKS(upload(ctx, D.kb, kb_all));
        CKS(upload(ctx, D.e_cap, e_cap));
        CK(launch_mirror(D, ctx->work));   // derived from x
        CKS(dev_alloc(ctx, ctx->cap_stats, CAP_STAT_DOUBLES * caps.size()));
        if (any_cells) {
            D.n_cells = cell_off;
            CKS(dev_alloc(ctx, D.cell_count, (size_t)cell_off));
            CKS(dev_alloc(ctx, D.cell_items, (size_t)cell_off * CELL_CAP));
            CKS(dev_alloc(ctx, D.cell_vid, (size_t)cell_off * CELL_CAP));
            CKS(dev_alloc(ctx, D.near, caps.size() * NEAR_STRIDE));
        }
    }
    // slab decomposition: every ghost plane of every slab, from the slab
    // that owns its global x
    if (ctx->slabs.S > 1) {
        const auto& P = ctx->slabs;
        std::vector<int4> pairs;
        for (int m = 0; m < P.S; ++m) {
            const ibl_slab& a = P.sl[m];
            const int w = a.x1 - a.x0;
            for (int l = 0; l < a.lo + w + a.hi; ++l) {
                if (l >= a.lo && l < a.lo + w) continue;
                int gx = a.x0 - a.lo + l;
                gx = ((gx % P.nx) + P.nx) % P.nx;
                int src = -1;
                for (int t = 0; t < P.S; ++t)
                    if (gx >= P.sl[t].x0 && gx < P.sl[t].x1) src = t;
                if (src < 0 || src == m) return fail(ctx, IBL_ERR_ARG, "slab plan: a ghost plane has no other owner");
                const ibl_slab& b = P.sl[src];
                pairs.push_back(make_int4(m, l + ctx->hmem[m].px, src, gx - b.x0 + b.lo + ctx->hmem[src].px));
            }
        }
        for (int m = 1; m < nm; ++m)
            if (ctx->hmem[m].NY != ctx->hmem[0].NY || ctx->hmem[m].NZ != ctx->hmem[0].NZ)
                return fail(ctx, IBL_ERR_ARG, "slab members differ in y or z");
        D.n_halo = (int)pairs.size();
        CKS(dev_alloc(ctx, D.halo, pairs.size()));
        CKS(upload(ctx, D.halo, pairs));
        if (nm == P.S + 1 && ctx->members[P.S].whole_view) {
            std::vector<int> of(P.nx, 0);
            std::vector<int4> tab(P.S);
            for (int m = 0; m < P.S; ++m) {
                const ibl_slab& b = P.sl[m];
                for (int x = b.x0; x < b.x1; ++x) of[x] = m;
                tab[m] = make_int4(b.x0, b.x1, b.lo, b.hi);
            }
            int* d_of = nullptr;
            int4* d_tab = nullptr;
            CKS(dev_alloc(ctx, d_of, of.size()));
            CKS(dev_alloc(ctx, d_tab, tab.size()));
            CKS(upload(ctx, d_of, of));
            CKS(upload(ctx, d_tab, tab));
            D.slab_of = d_of;
            D.slab_tab = d_tab;
            D.slab_w = P.S;
            D.n_slabs = P.S;
        }
    }
    D.h_mem = ctx->hmem.data();
    CKS(dev_alloc(ctx, D.mem, (size_t)nm));
    CKS(upload(ctx, D.mem, ctx->hmem));
    // initial populations
    for (int mi = 0; mi < nm; ++mi) {
        const MemberHost& M = ctx->members[mi];
        if (M.whole_view) continue;
        float* drho = nullptr;
        float* du = nullptr;
        if (!M.init_rho.empty()) { CK(cudaMalloc((void**)&drho, sizeof(float) * M.init_rho.size())); }
        if (!M.init_u.empty()) { CK(cudaMalloc((void**)&du, sizeof(float) * M.init_u.size())); }
        if (drho) CK(cudaMemcpyAsync(drho, M.init_rho.data(), sizeof(float) * M.init_rho.size(), cudaMemcpyHostToDevice, ctx->work));
        if (du) CK(cudaMemcpyAsync(du, M.init_u.data(), sizeof(float) * M.init_u.size(), cudaMemcpyHostToDevice, ctx->work));
        CK(launch_init_member(D, mi, drho, du, ctx->work));
        CK(cudaStreamSynchronize(ctx->work));
        if (drho) cudaFree(drho);
        if (du) cudaFree(du);
    }
    D.lattice_path = ctx->lattice_path;
    if (D.chunks) CKS(prepare_staged(ctx));
    ctx->h_counters.assign(nm, 0);
    ctx->h_status.assign(nm, 0);
    CK(cudaStreamSynchronize(ctx->work));
    ctx->finalized = true;
    return IBL_OK;
}

enum { TK_LBM = 0, TK_BFL = 1, TK_IB = 2, TK_STRUCT = 3 };

// What the discrete adjoint needs from one forward step, written while the
// step runs: (rho, u) and the IB force of every fluid node before the
// collision, d(value)/dq of every wall link, rho of every face node, and the
// vertex positions and velocities at the start of the step.  Any pointer may
// be null.
struct StepTape {
    float4* rhou = nullptr;
    float4* F = nullptr;
    float* dvdq = nullptr;
    float* rho = nullptr;
    double* x = nullptr;
    double* v = nullptr;
};

struct Mark {
    int kind;
    cudaEvent_t a, b;
};

// One time step.  Stream `work`: step begin, geometry, shell moments, the
// marker stencils, then the lattice step, the wall fill and the faces.
// (Timing mode runs every phase on `work`, one after another.)
// Stream `work3`: the probe stencils, beside the marker stencils and the
// lattice step.  Stream `work2`: after the geometry, repulsion and hinge
// forces (beside the IB pass); after the markers and the probes, the
// structure update (beside the lattice step).  The update touches no lattice
// data and the lattice step no structure data.
ibl_status enqueue_step(ibl_ctx* ctx, int parity, std::vector<Mark>* marks, const StepTape* tp = nullptr) {
    DevState& D = ctx->dev;
    cudaStream_t s = ctx->work, s2 = ctx->work2, s3 = ctx->work3;
    if (tp && tp->x && D.n_verts > 0) {
        CK(cudaMemcpyAsync(tp->x, D.x, sizeof(double) * 3 * (size_t)D.n_verts, cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(tp->v, D.vel, sizeof(double) * 3 * (size_t)D.n_verts, cudaMemcpyDeviceToDevice, s));
    }
    cudaEvent_t e0 = nullptr;
    auto begin = [&](cudaStream_t st) -> ibl_status {
        if (!marks) return IBL_OK;
        CK(cudaEventCreate(&e0));
        CK(cudaEventRecord(e0, st));
        return IBL_OK;
    };
    auto end = [&](int kind, cudaStream_t st) -> ibl_status {
        if (!marks) return IBL_OK;
        cudaEvent_t e1;
        CK(cudaEventCreate(&e1));
        CK(cudaEventRecord(e1, st));
        marks->push_back(Mark{kind, e0, e1});
        return IBL_OK;
    };
    CK(launch_step_begin(D, s));
    const bool caps = D.n_caps > 0;
    if (caps && marks) {
        // timing mode: the phases run one after another on one stream, so
        // that each phase's events time it alone
        CKS(begin(s));
        CK(launch_geometry(D, 0, s));
        CK(launch_shell(D, parity, s));
        CK(launch_markers(D, s));
        CK(launch_probes(D, s));
        CK(launch_fib_scatter(D, s));
        CKS(end(TK_IB, s));
        CKS(begin(s));
        CK(launch_repulsion(D, s));
        CK(launch_edges(D, s));
        CK(launch_update(D, s));
        CKS(end(TK_STRUCT, s));
    } else if (caps) {
        CK(launch_geometry(D, 0, s));
        CK(cudaEventRecord(ctx->ev_fork, s));
        CK(launch_shell(D, parity, s));
        CK(cudaEventRecord(ctx->ev_shell, s));
        CK(launch_markers(D, s));
        CK(cudaEventRecord(ctx->ev_ib, s));
        CK(launch_fib_scatter(D, s));
        CK(cudaStreamWaitEvent(s3, ctx->ev_shell, 0));
        CK(launch_probes(D, s3));
        CK(cudaEventRecord(ctx->ev_probes, s3));
        CK(cudaStreamWaitEvent(s2, ctx->ev_fork, 0));
        CK(launch_repulsion(D, s2));
        CK(launch_edges(D, s2));
        CK(cudaStreamWaitEvent(s2, ctx->ev_ib, 0));
        CK(cudaStreamWaitEvent(s2, ctx->ev_probes, 0));
        CK(launch_update(D, s2));
    }
    CKS(begin(s));
    if (!tp && D.lattice_path == 1 && D.chunks && D.bulk_blocks_per_sm > 0) {
        // staged kernel over the interior chunks, the register kernel over
        // the wrap-plane nodes only
        CK(launch_lbm_bulk(D, parity, s));
        DevState Db = D;
        Db.lbm_blocks = 0;
        Db.grid_lbm = 0;
        CK(launch_lbm(Db, parity, s));
    } else {
        CK(launch_lbm(D, parity, s, tp ? tp->rhou : nullptr, tp ? tp->F : nullptr));
    }
    CKS(end(TK_LBM, s));
    CKS(begin(s));
    CK(launch_walls(D, parity, s, tp ? tp->dvdq : nullptr, tp ? tp->rho : nullptr));
    CK(launch_halo(D, s));
    CKS(end(TK_BFL, s));
    if (caps && !marks) {
        CK(cudaEventRecord(ctx->ev_join, s2));
        CK(cudaStreamWaitEvent(s, ctx->ev_join, 0));
    }
    if (caps) CK(launch_status_spread(D, s));
    return IBL_OK;
}

ibl_status capture_graph(ibl_ctx* ctx, int parity) {
    if (ctx->graph[parity]) return IBL_OK;
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(ctx->work, cudaStreamCaptureModeThreadLocal));
    ibl_status st = enqueue_step(ctx, parity, nullptr);
    cudaError_t e = cudaStreamEndCapture(ctx->work, &g);
    if (st != IBL_OK) { if (g) cudaGraphDestroy(g); return st; }
    CK(e);
    // kernel launches per step = kernel nodes of the captured step
    size_t n_nodes = 0;
    int n_kernels = 0;
    if (cudaGraphGetNodes(g, nullptr, &n_nodes) == cudaSuccess && n_nodes > 0) {
        std::vector<cudaGraphNode_t> nodes(n_nodes);
        if (cudaGraphGetNodes(g, nodes.data(), &n_nodes) == cudaSuccess)
            for (size_t i = 0; i < n_nodes; ++i) {
                cudaGraphNodeType t;
                if (cudaGraphNodeGetType(nodes[i], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++n_kernels;
            }
    }
    ctx->graph_kernels[parity] = n_kernels;
    e = cudaGraphInstantiate(&ctx->graph[parity], g, 0);
    cudaGraphDestroy(g);
    CK(e);
    return IBL_OK;
}

ibl_status sync_host_state(ibl_ctx* ctx) {
    const int nm = ctx->dev.n_members;
    CK(cudaMemcpyAsync(ctx->h_counters.data(), ctx->dev.counters, sizeof(int) * nm, cudaMemcpyDeviceToHost, ctx->work));
    std::vector<uint32_t> pending(nm);
    CK(cudaMemcpyAsync(ctx->h_status.data(), ctx->dev.status, sizeof(uint32_t) * nm, cudaMemcpyDeviceToHost, ctx->work));
    CK(cudaMemcpyAsync(pending.data(), ctx->dev.status_new, sizeof(uint32_t) * nm, cudaMemcpyDeviceToHost, ctx->work));
    CK(cudaStreamSynchronize(ctx->work));
    for (int m = 0; m < nm; ++m) ctx->h_status[m] |= pending[m];
    return IBL_OK;
}

MemberHost* member0(ibl_ctx* ctx) { return ctx->members.empty() ? nullptr : &ctx->members[0]; }

ibl_status read_fields_member(ibl_ctx* ctx, int m, float* rho, float* u, float* g, int on_device) {
    if (m < 0 || m >= (int)ctx->members.size()) return fail(ctx, IBL_ERR_ARG, "member out of range");
    if (ctx->members[m].whole_view) return fail(ctx, IBL_ERR_ARG, "the whole-lattice member of a slab context holds no populations");
    CKS(finalize(ctx));
    CKS(enter(ctx));
    const MemberDev& md = ctx->hmem[m];
    const size_t Nu = (size_t)md.nx * md.ny * md.nz;
    const int cnt = ctx->h_counters[m];
    const int parity = cnt & 1;
    // page-locked host buffers that the device can address (every
    // page-locked allocation, with unified addressing) take the read kernel's
    // output directly: no staging buffer, no copy
    auto mapped = [](void* p, void** dp) -> bool {
        *dp = nullptr;
        if (!p) return true;
        cudaPointerAttributes a;
        if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        *dp = a.devicePointer;
        return a.type == cudaMemoryTypeHost && a.devicePointer != nullptr;
    };
    void *mr = nullptr, *mu = nullptr, *mg = nullptr;
    const bool direct = !on_device && mapped(rho, &mr) && mapped(u, &mu) && mapped(g, &mg);
    if (on_device) {
        CK(launch_read(ctx->dev, m, parity, rho, u, g, ctx->work));
    } else if (direct) {
        CK(launch_read(ctx->dev, m, parity, (float*)mr, (float*)mu, (float*)mg, ctx->work));
        CK(cudaStreamSynchronize(ctx->work));
    } else {
        // one device staging buffer per context, allocated by the first host
        // read and grown when a larger one is needed
        const size_t need = sizeof(float) * Nu * ((rho ? 1 : 0) + (u ? 3 : 0) + (g ? 19 : 0));
        if (need > ctx->stage_bytes) {
            CK(cudaStreamSynchronize(ctx->work));
            if (ctx->stage) cudaFree(ctx->stage);
            ctx->stage = nullptr;
            ctx->stage_bytes = 0;
            const cudaError_t e = cudaMalloc((void**)&ctx->stage, need);
            if (e != cudaSuccess) {
                cudaGetLastError();
                ctx->stage = nullptr;
                return fail(ctx, IBL_ERR_OOM, "read staging buffer: cudaMalloc of " + std::to_string(need) + " bytes failed");
            }
            ctx->stage_bytes = need;
        }
        float* dr = rho ? ctx->stage : nullptr;
        float* du = u ? ctx->stage + (rho ? Nu : 0) : nullptr;
        float* dg = g ? ctx->stage + (rho ? Nu : 0) + (u ? 3 * Nu : 0) : nullptr;
        CK(launch_read(ctx->dev, m, parity, dr, du, dg, ctx->work));
        if (rho) CK(cudaMemcpyAsync(rho, dr, sizeof(float) * Nu, cudaMemcpyDeviceToHost, ctx->work));
        if (u) CK(cudaMemcpyAsync(u, du, sizeof(float) * 3 * Nu, cudaMemcpyDeviceToHost, ctx->work));
        if (g) CK(cudaMemcpyAsync(g, dg, sizeof(float) * 19 * Nu, cudaMemcpyDeviceToHost, ctx->work));
        CK(cudaStreamSynchronize(ctx->work));
    }
    CKS(leave(ctx));
    return IBL_OK;
}

// The member whose capsules member m's capsule calls address: in a slab
// context the capsules live in its whole-lattice member.
int caps_member(const ibl_ctx* ctx, int m) {
    const int n = (int)ctx->members.size();
    if (ctx->slabs.S > 1 && m == 0 && n == ctx->slabs.S + 1 && ctx->members[n - 1].whole_view) return n - 1;
    return m;
}

// The whole lattice of a slab context: each slab's owned planes, read from
// its member into host buffers.
ibl_status read_fields_slabs(ibl_ctx* ctx, float* rho, float* u, float* g, int on_device) {
    if (on_device) return fail(ctx, IBL_ERR_ARG, "a slab context reads the whole lattice into host buffers only");
    const auto& P = ctx->slabs;
    const int ny = ctx->members[0].desc.ny, nz = ctx->members[0].desc.nz;
    const size_t Ng = (size_t)P.nx * ny * nz;
    for (int m = 0; m < P.S; ++m) {
        const ibl_slab& b = P.sl[m];
        const int nxs = ctx->members[m].desc.nx;
        const size_t Ns = (size_t)nxs * ny * nz;
        std::vector<float> r(rho ? Ns : 0), v(u ? 3 * Ns : 0), q(g ? 19 * Ns : 0);
        CKS(read_fields_member(ctx, m, rho ? r.data() : nullptr, u ? v.data() : nullptr, g ? q.data() : nullptr, 0));
        for (int z = 0; z < nz; ++z)
            for (int y = 0; y < ny; ++y)
                for (int x = b.x0; x < b.x1; ++x) {
                    const size_t ln = (x - b.x0 + b.lo) + (size_t)nxs * (y + (size_t)ny * z);
                    const size_t gn = x + (size_t)P.nx * (y + (size_t)ny * z);
                    if (rho) rho[gn] = r[ln];
                    if (u)
                        for (int c = 0; c < 3; ++c) u[3 * gn + c] = v[3 * ln + c];
                    if (g)
                        for (int k = 0; k < 19; ++k) g[k * Ng + gn] = q[k * Ns + ln];
                }
    }
    return IBL_OK;
}

ibl_status read_capsule_member(ibl_ctx* ctx, int m, int id, ibl_capsule_stats* st, double* verts_out) {
    if (m < 0 || m >= (int)ctx->members.size()) return fail(ctx, IBL_ERR_ARG, "member out of range");
    CKS(finalize(ctx));
    if (id < 0 || id >= (int)ctx->member_caps[m].size()) return fail(ctx, IBL_ERR_ARG, "capsule id out of range");
    const int cap = ctx->member_caps[m][id];
    const CapsuleRestHost& R = ctx->rest[cap];
    CKS(enter(ctx));
    std::vector<double> X(3 * (size_t)R.nv), V(3 * (size_t)R.nv);
    CK(cudaMemcpyAsync(X.data(), ctx->dev.x + 3 * (size_t)R.v_begin, sizeof(double) * X.size(), cudaMemcpyDeviceToHost, ctx->work));
    CK(cudaMemcpyAsync(V.data(), ctx->dev.vel + 3 * (size_t)R.v_begin, sizeof(double) * V.size(), cudaMemcpyDeviceToHost, ctx->work));
    CK(cudaStreamSynchronize(ctx->work));
    CKS(leave(ctx));
    if (verts_out) std::memcpy(verts_out, X.data(), sizeof(double) * X.size());
    if (st) {
        const std::vector<int>& tris = ctx->members[m].caps[id].tris;
        MeshSums ms = mesh_sums(X.data(), R.nv, tris.data(), R.nt);
        std::memset(st, 0, sizeof(*st));
        st->centroid[0] = ms.cen.x; st->centroid[1] = ms.cen.y; st->centroid[2] = ms.cen.z;
        st->volume = ms.V;
        st->area = ms.S;
        st->dS = (ms.S - R.S0) / R.S0;
        double ev[3];
        sym3_eigen(ms.M2, ev);
        for (int a = 0; a < 3; ++a) st->semi_axes[a] = std::sqrt(std::max(5.0 * ev[a] / ms.V, 0.0));
        st->taylor_D = (st->semi_axes[2] - st->semi_axes[0]) / (st->semi_axes[2] + st->semi_axes[0]);
        double mx = 0.0;
        for (int e = 0; e < R.ne; ++e) {
            const int a = R.edges[2 * e], b = R.edges[2 * e + 1];
            const double dx = X[3 * a] - X[3 * b], dy = X[3 * a + 1] - X[3 * b + 1], dz = X[3 * a + 2] - X[3 * b + 2];
            mx = std::max(mx, std::sqrt(dx * dx + dy * dy + dz * dz) / R.l0[e]);
        }
        st->max_stretch = R.rigid ? 1.0 : mx;
        for (int v = 0; v < R.nv; ++v)
            for (int a = 0; a < 3; ++a) st->velocity[a] += V[3 * v + a] / R.nv;
        st->damaged = (ctx->h_status[m] & ST_DAMAGED) ? 1 : 0;
    }
    return IBL_OK;
}


// ---------------------------------------------------------------------------
// State snapshot: everything a later step reads that the steps themselves
// change.  Between steps f_ib, the IB tag bits, the force and normal/area
// accumulators are zero or recomputed, so they are not part of it.
// ---------------------------------------------------------------------------
struct StateHeader {
    char magic[8];
    uint32_t version, storage;
    uint64_t f_bytes;
    int32_t n_members, n_caps, n_verts, reserved;
    int64_t t;
};

struct StateSection {
    void* dev;
    size_t bytes;
};

std::vector<StateSection> state_sections(ibl_ctx* ctx) {
    const DevState& D = ctx->dev;
    const size_t nm = (size_t)D.n_members, nv3 = 3 * (size_t)D.n_verts;
    std::vector<StateSection> s = {{D.f, D.f_bytes},
                                   {D.status, sizeof(uint32_t) * nm},
                                   {D.status_new, sizeof(uint32_t) * nm},
                                   {D.counters, sizeof(int) * nm}};
    if (D.n_caps > 0) {
        s.push_back({D.caps, sizeof(CapsuleDev) * (size_t)D.n_caps});
        s.push_back({D.x, sizeof(double) * nv3});
        s.push_back({D.x_prev, sizeof(double) * nv3});
        s.push_back({D.vel, sizeof(double) * nv3});
    }
    return s;
}

StateHeader state_header(ibl_ctx* ctx) {
    StateHeader h{};
    std::memcpy(h.magic, "IBLSTAT", 8);
    h.version = 1;
    h.storage = (uint32_t)ctx->storage;
    h.f_bytes = ctx->dev.f_bytes;
    h.n_members = ctx->dev.n_members;
    h.n_caps = ctx->dev.n_caps;
    h.n_verts = ctx->dev.n_verts;
    h.t = ctx->t;
    return h;
}

size_t state_bytes(ibl_ctx* ctx) {
    size_t n = sizeof(StateHeader);
    for (const StateSection& s : state_sections(ctx)) n += s.bytes;
    return n;
}

ibl_status new_ctx(void* stream, ibl_ctx** out) {
    ibl_ctx* ctx = new (std::nothrow) ibl_ctx();
    if (!ctx) return fail(nullptr, IBL_ERR_OOM, "host allocation failed");
    ctx->user_stream = (cudaStream_t)stream;
    cudaError_t e = cudaGetDevice(&ctx->device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->work, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->work2, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->work3, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_shell, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_probes, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_ib, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_in, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_out, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        ibl_destroy(ctx);   // releases whatever was created
        return fail(nullptr, IBL_ERR_CUDA, std::string("stream/event creation failed: ") + cudaGetErrorString(e));
    }
    *out = ctx;
    return IBL_OK;
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

ibl_status ibl_create(const ibl_lattice_desc* desc, void* cuda_stream, ibl_ctx** out) {
    if (!desc || !out) return fail(nullptr, IBL_ERR_ARG, "null argument");
    *out = nullptr;
    if (desc->nx < 3 || desc->ny < 3 || desc->nz < 1 || (desc->nz < 3 && !desc->periodic[2]))
        return fail(nullptr, IBL_ERR_ARG, "lattice dimensions too small (non-periodic axes need >= 3 nodes)");
    if (desc->nx < 3 && !desc->periodic[0]) return fail(nullptr, IBL_ERR_ARG, "lattice dimensions too small");
    if (!(desc->tau > 0.5)) return fail(nullptr, IBL_ERR_ARG, "tau must exceed 1/2");
    if (desc->storage < 0 || desc->storage > 2) return fail(nullptr, IBL_ERR_ARG, "unknown storage");
    ibl_ctx* ctx = nullptr;
    ibl_status st = new_ctx(cuda_stream, &ctx);
    if (st != IBL_OK) return st;
    ctx->storage = desc->storage;
    ctx->members.resize(1);
    ctx->members[0].desc = *desc;
    const size_t N = (size_t)desc->nx * desc->ny * desc->nz;
    ctx->members[0].tag.assign(N, 0);
    *out = ctx;
    return IBL_OK;
}

ibl_status ibl_set_geometry(ibl_ctx* ctx, const uint8_t* cell_tag, const ibl_wall_link* links, size_t n_links) {
    if (!ctx) return fail(nullptr, IBL_ERR_ARG, "null context");
    if (ctx->finalized) return fail(ctx, IBL_ERR_STATE, "geometry is fixed once the context has been stepped or read");
    if (ctx->members.size() != 1) return fail(ctx, IBL_ERR_STATE, "an ensemble takes its geometry from its members");
    MemberHost& M = ctx->members[0];
    const size_t N = M.tag.size();
    if (!cell_tag || (n_links && !links)) return fail(ctx, IBL_ERR_ARG, "null geometry array");
    {
        // eight tags per word: any bit but the lowest of a byte is set
        size_t n = 0;
        for (; n + 8 <= N; n += 8) {
            uint64_t w;
            std::memcpy(&w, cell_tag + n, 8);
            if (w & 0xfefefefefefefefeull) break;
        }
        for (; n < N; ++n)
            if (cell_tag[n] > 1) return fail(ctx, IBL_ERR_ARG, "cell_tag values must be 0 (fluid) or 1 (solid)");
    }
    M.tag.assign(cell_tag, cell_tag + N);
    M.links.assign(links, links + n_links);
    return IBL_OK;
}

static size_t face_count(const ibl_lattice_desc& d, int face) {
    return face < 2 ? (size_t)d.ny * d.nz : (face < 4 ? (size_t)d.nx * d.nz : (size_t)d.nx * d.ny);
}

ibl_status ibl_set_inlet_velocity(ibl_ctx* ctx, int32_t face, const float* u_xyz) {
    if (!ctx) return fail(nullptr, IBL_ERR_ARG, "null context");
    if (ctx->finalized) return fail(ctx, IBL_ERR_STATE, "faces are fixed once the context has been stepped or read");
    if (face < 0 || face > 5 || !u_xyz) return fail(ctx, IBL_ERR_ARG, "bad face or null velocity");
    MemberHost* M = member0(ctx);
    if (M->desc.periodic[face / 2]) return fail(ctx, IBL_ERR_ARG, "face lies on a periodic axis");
    const size_t n = face_count(M->desc, face);
    M->face_kind[face] = IBL_FACE_VELOCITY;
    M->face_vel[face].assign(u_xyz, u_xyz + 3 * n);
    return IBL_OK;
}

ibl_status ibl_set_outlet_pressure(ibl_ctx* ctx, int32_t face, double rho_out) {
    if (!ctx) return fail(nullptr, IBL_ERR_ARG, "null context");
    if (ctx->finalized) return fail(ctx, IBL_ERR_STATE, "faces are fixed once the context has been stepped or read");
    if (face < 0 || face > 5 || !(rho_out > 0)) return fail(ctx, IBL_ERR_ARG, "bad face or density");
    MemberHost* M = member0(ctx);
    if (M->desc.periodic[face / 2]) return fail(ctx, IBL_ERR_ARG, "face lies on a periodic axis");
    M->face_kind[face] = IBL_FACE_PRESSURE;
    M->face_rho[face] = rho_out;
    M->face_vel[face].clear();
    return IBL_OK;
}

ibl_status ibl_init_equilibrium(ibl_ctx* ctx, const float* rho, const float* u) {
    if (!ctx) return fail(nullptr, IBL_ERR_ARG, "null context");
    if (ctx->finalized) return fail(ctx, IBL_ERR_STATE, "initial state is fixed once the context has been stepped or read");
    MemberHost* M = member0(ctx);
    const size_t N = M->tag.size();
    if (rho) M->init_rho.assign(rho, rho + N); else M->init_rho.clear();
    if (u) M->init_u.assign(u, u + 3 * N); else M->init_u.clear();
    return IBL_OK;
}

ibl_status ibl_add_capsule(ibl_ctx* ctx, const double* verts, int32_t nv, const int32_t* tris, int32_t nt,
                           const double* vel0, const ibl_capsule_params* params, int32_t* id_out) {
    if (!ctx) return fail(nullptr, IBL_ERR_ARG, "null context");
    if (ctx->finalized) return fail(ctx, IBL_ERR_STATE, "capsules must be added before the first step or read");
    if (!verts || !tris || !params || nv < 4 || nt < 4) return fail(ctx, IBL_ERR_ARG, "bad capsule arguments");
    if (!params->rigid && !(params->Ca > 0)) return fail(ctx, IBL_ERR_ARG, "a soft capsule needs Ca > 0");
    if (!(params->density_ratio > 0)) return fail(ctx, IBL_ERR_ARG, "density_ratio must be positive");
    MemberHost* M = member0(ctx);
    CapsuleHost ch;
    ch.X.assign(verts, verts + 3 * (size_t)nv);
    ch.tris.assign(tris, tris + 3 * (size_t)nt);
    if (vel0) for (int a = 0; a < 3; ++a) ch.vel0[a] = vel0[a];
    ch.p = *params;
    // the cheap check here; closure and orientation when the context is set
    // up, where the hinges are built on host threads
    for (int t = 0; t < nt; ++t) {
        const int a = tris[3 * t], b = tris[3 * t + 1], c = tris[3 * t + 2];
        if (a < 0 || b < 0 || c < 0 || a >= nv || b >= nv || c >= nv || a == b || b == c || a == c)
            return fail(ctx, IBL_ERR_ARG, "capsule mesh: triangle " + std::to_string(t) + " has an invalid vertex index");
    }
    M->caps.push_back(std::move(ch));
    if (id_out) *id_out = (int32_t)M->caps.size() - 1;
    return IBL_OK;
}

ibl_status ibl_step(ibl_ctx* ctx, int32_t n_steps, int32_t* steps_done) {
    if (!ctx) return fail(nullptr, IBL_ERR_ARG, "null context");
    if (n_steps < 0) return fail(ctx, IBL_ERR_ARG, "negative step count");
    CKS(finalize(ctx));
    const int before = ctx->h_counters[0];
    CKS(enter(ctx));
    std::vector<Mark> marks;
    for (int s = 0; s < n_steps; ++s) {
        const int parity = (int)(ctx->t & 1);
        if (ctx->timing) {
            CKS(enqueue_step(ctx, parity, &marks));
        } else if (ctx->use_graphs) {
            CKS(capture_graph(ctx, parity));
            CK(cudaGraphLaunch(ctx->graph[parity], ctx->work));
        } else {
            CKS(enqueue_step(ctx, parity, nullptr));
        }
        ctx->t += 1;
    }
    CKS(sync_host_state(ctx));
    CKS(leave(ctx));
    if (ctx->timing) {
        for (double& v : ctx->ktime) v = 0.0;
        for (const Mark& mk : marks) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, mk.a, mk.b);
            ctx->ktime[mk.kind] += ms;
            cudaEventDestroy(mk.a);
            cudaEventDestroy(mk.b);
        }
    }
    if (steps_done) *steps_done = ctx->h_counters[0] - before;
    uint32_t any = 0;
    for (uint32_t s : ctx->h_status) any |= s;
    if (any & ST_NONFINITE) return fail(ctx, IBL_ERR_NONFINITE, "a capsule vertex became non-finite");
    if (any & ST_DAMAGED) return fail(ctx, IBL_ERR_DAMAGED, "a capsule edge reached twice its rest length");
    if (any & ST_OVERFLOW) return fail(ctx, IBL_ERR_ARG, "repulsion cell list overflow (markers too dense)");
    if (any & ST_TIMEOUT) return fail(ctx, IBL_ERR_TIMEOUT, "a bounded wait of the staged lattice kernel gave up");
    return IBL_OK;
}

ibl_status ibl_read_fields(ibl_ctx* ctx, float* rho, float* u, int32_t on_device) {
    if (!ctx) return fail(nullptr, IBL_ERR_ARG, "null context");
    if (ctx->slabs.S > 1) return read_fields_slabs(ctx, rho, u, nullptr, on_device);
    return read_fields_member(ctx, 0, rho, u, nullptr, on_device);
}

ibl_status ibl_read_populations(ibl_ctx* ctx, float* g, int32_t on_device) {
    if (!ctx) return fail(nullptr, IBL_ERR_ARG, "null context");
    if (!g) return fail(ctx, IBL_ERR_ARG, "null output");
    if (ctx->slabs.S > 1) return read_fields_slabs(ctx, nullptr, nullptr, g, on_device);
    return read_fields_member(ctx, 0, nullptr, nullptr, g, on_device);
}

ibl_status ibl_read_capsule(ibl_ctx* ctx, int32_t id, ibl_capsule_stats* stats, double* verts_out) {
    if (!ctx) return fail(nullptr, IBL_ERR_ARG, "null context");
    return read_capsule_member(ctx, caps_member(ctx, 0), id, stats, verts_out);
}

ibl_status ibl_read_capsules(ibl_ctx* ctx, int32_t member, ibl_capsule_stats* stats, int32_t n) {
    if (!ctx || !stats) return fail(ctx, IBL_ERR_ARG, "null argument");
    if (member < 0 || member >= (int)ctx->members.size()) return fail(ctx, IBL_ERR_ARG, "member out of range");
    CKS(finalize(ctx));
    member = caps_member(ctx, member);
    const std::vector<int>& ids = ctx->member_caps[member];
    if (n != (int32_t)ids.size())
        return fail(ctx, IBL_ERR_ARG, "member " + std::to_string(member) + " holds " + std::to_string(ids.size()) +
                                          " capsules");
    if (n == 0) return IBL_OK;
    const int c0 = ids[0];
    CKS(enter(ctx));
    CK(launch_capsule_stats(ctx->dev, c0, n, ctx->cap_stats, ctx->work));
    ctx->h_cap_stats.resize((size_t)CAP_STAT_DOUBLES * n);
    CK(cudaMemcpyAsync(ctx->h_cap_stats.data(), ctx->cap_stats + (size_t)c0 * CAP_STAT_DOUBLES,
                       sizeof(double) * CAP_STAT_DOUBLES * n, cudaMemcpyDeviceToHost, ctx->work));
    CK(cudaStreamSynchronize(ctx->work));
    CKS(leave(ctx));
    const bool damaged = (ctx->h_status[member] & ST_DAMAGED) != 0;
    for (int i = 0; i < n; ++i) {
        const double* o = ctx->h_cap_stats.data() + (size_t)CAP_STAT_DOUBLES * i;
        const CapsuleRestHost& R = ctx->rest[c0 + i];
        ibl_capsule_stats* st = stats + i;
        std::memset(st, 0, sizeof(*st));
        const double V = o[0];
        const double cr[3] = {o[2] / V, o[3] / V, o[4] / V};
        for (int a = 0; a < 3; ++a) st->centroid[a] = o[15 + a] + cr[a];
        st->volume = V;
        st->area = o[1];
        st->dS = (o[1] - R.S0) / R.S0;
        // second moments about the centroid
        const double M[6] = {o[5] - V * cr[0] * cr[0], o[6] - V * cr[1] * cr[1], o[7] - V * cr[2] * cr[2],
                             o[8] - V * cr[0] * cr[1], o[9] - V * cr[0] * cr[2], o[10] - V * cr[1] * cr[2]};
        double ev[3];
        sym3_eigen(M, ev);
        for (int a = 0; a < 3; ++a) st->semi_axes[a] = std::sqrt(std::max(5.0 * ev[a] / V, 0.0));
        st->taylor_D = (st->semi_axes[2] - st->semi_axes[0]) / (st->semi_axes[2] + st->semi_axes[0]);
        st->max_stretch = R.rigid ? 1.0 : o[14];
        for (int a = 0; a < 3; ++a) st->velocity[a] = o[11 + a] / R.nv;
        st->damaged = damaged ? 1 : 0;
    }
    return IBL_OK;
}

ibl_status ibl_read_capsule_state(ibl_ctx* ctx, int32_t id, double* x, double* x_prev, double* vel, double* force) {
    if (!ctx) return fail(nullptr, IBL_ERR_ARG, "null context");
    CKS(finalize(ctx));
    const int cm = caps_member(ctx, 0);
    if (id < 0 || id >= (int)ctx->member_caps[cm].size()) return fail(ctx, IBL_ERR_ARG, "capsule id out of range");
    const CapsuleRestHost& R = ctx->rest[ctx->member_caps[cm][id]];
    const size_t n3 = 3 * (size_t)R.nv, off = 3 * (size_t)R.v_begin;
    CKS(enter(ctx));
    std::vector<float> F(4 * (size_t)R.nv);
    if (x) CK(cudaMemcpyAsync(x, ctx->dev.x + off, sizeof(double) * n3, cudaMemcpyDeviceToHost, ctx->work));
    if (x_prev) CK(cudaMemcpyAsync(x_prev, ctx->dev.x_prev + off, sizeof(double) * n3, cudaMemcpyDeviceToHost, ctx->work));
    if (vel) CK(cudaMemcpyAsync(vel, ctx->dev.vel + off, sizeof(double) * n3, cudaMemcpyDeviceToHost, ctx->work));
    if (force)
        CK(cudaMemcpyAsync(F.data(), ctx->dev.force + 4 * (size_t)R.v_begin, sizeof(float) * F.size(),
                           cudaMemcpyDeviceToHost, ctx->work));
    CK(cudaStreamSynchronize(ctx->work));
    CKS(leave(ctx));
    if (force)
        for (size_t v = 0; v < (size_t)R.nv; ++v)
            for (int a = 0; a < 3; ++a) force[3 * v + a] = F[4 * v + a];
    return IBL_OK;
}

ibl_status ibl_ensemble_create(ibl_ctx* const* members, int32_t n, void* cuda_stream, ibl_ctx** out) {
    if (!members || !out || n < 1 || n > MAX_MEMBERS) return fail(nullptr, IBL_ERR_ARG, "bad ensemble arguments");
    *out = nullptr;
    int storage = -1;
    for (int i = 0; i < n; ++i) {
        if (!members[i]) return fail(nullptr, IBL_ERR_ARG, "null member");
        if (members[i]->finalized) return fail(nullptr, IBL_ERR_STATE, "ensemble members must not have been stepped or read");
        if (storage >= 0 && members[i]->storage != storage) return fail(nullptr, IBL_ERR_ARG, "members use different storage");
        storage = members[i]->storage;
    }
    ibl_ctx* ctx = nullptr;
    ibl_status st = new_ctx(cuda_stream, &ctx);
    if (st != IBL_OK) return st;
    ctx->storage = storage;
    for (int i = 0; i < n; ++i)
        for (const MemberHost& M : members[i]->members) ctx->members.push_back(M);
    if ((int)ctx->members.size() > MAX_MEMBERS) {
        ibl_destroy(ctx);
        return fail(nullptr, IBL_ERR_ARG, "too many members");
    }
    *out = ctx;
    return IBL_OK;
}

ibl_status ibl_slab_plan(int32_t nx, int32_t periodic_x, int32_t n_slabs, int32_t halo, const double* plane_weight,
                         ibl_slab* out) {
    if (!out) return fail(nullptr, IBL_ERR_ARG, "null output");
    std::vector<ibl_slab> sl;
    std::string why;
    if (!plan_slabs(nx, periodic_x != 0, n_slabs, halo, plane_weight, sl, why)) return fail(nullptr, IBL_ERR_ARG, why);
    std::copy(sl.begin(), sl.end(), out);
    return IBL_OK;
}

ibl_status ibl_slab_group_create(ibl_ctx* whole, int32_t n_slabs, int32_t halo, void* cuda_stream, ibl_ctx** out) {
    if (!whole || !out) return fail(nullptr, IBL_ERR_ARG, "null argument");
    *out = nullptr;
    if (whole->finalized) return fail(nullptr, IBL_ERR_STATE, "the whole lattice must not have been stepped or read");
    if (whole->members.size() != 1 || whole->slabs.S > 1)
        return fail(nullptr, IBL_ERR_STATE, "a slab context is cut from one lattice");
    const MemberHost& W = whole->members[0];
    if (halo < 4) return fail(nullptr, IBL_ERR_ARG, "halo must be at least 4 planes");
    if (n_slabs + (W.caps.empty() ? 0 : 1) > MAX_MEMBERS) return fail(nullptr, IBL_ERR_ARG, "too many slabs");
    const auto& d = W.desc;
    if ((long long)W.tag.size() != (long long)d.nx * d.ny * d.nz) return fail(nullptr, IBL_ERR_STATE, "geometry not set");
    // balance the slabs by fluid nodes per plane
    std::vector<double> wgt(d.nx, 0.0);
    for (size_t n = 0; n < W.tag.size(); ++n)
        if (W.tag[n] == 0) wgt[n % (size_t)d.nx] += 1.0;
    std::vector<ibl_slab> sl;
    std::string why;
    if (!plan_slabs(d.nx, d.periodic[0] != 0, n_slabs, halo, wgt.data(), sl, why)) return fail(nullptr, IBL_ERR_ARG, why);
    ibl_ctx* ctx = nullptr;
    ibl_status st = new_ctx(cuda_stream, &ctx);
    if (st != IBL_OK) return st;
    ctx->storage = whole->storage;
    ctx->members.resize(n_slabs);
    for (int m = 0; m < n_slabs; ++m)
        if (!crop_slab(W, sl[m], n_slabs, ctx->members[m], why)) {
            ibl_destroy(ctx);
            return fail(nullptr, IBL_ERR_ARG, why);
        }
    if (!W.caps.empty() && n_slabs > 1) {
        MemberHost V;
        V.desc = W.desc;
        V.tag = W.tag;
        V.caps = W.caps;
        V.whole_view = true;
        ctx->members.push_back(std::move(V));
    } else if (!W.caps.empty()) {
        ctx->members[0].caps = W.caps;
    }
    ctx->slabs.S = n_slabs;
    ctx->slabs.H = halo;
    ctx->slabs.nx = d.nx;
    ctx->slabs.per = d.periodic[0] ? 1 : 0;
    ctx->slabs.sl = sl;
    *out = ctx;
    return IBL_OK;
}

ibl_status ibl_slab_info(const ibl_ctx* ctx, int32_t* n_slabs, ibl_slab* out) {
    if (!ctx || !n_slabs) return fail(nullptr, IBL_ERR_ARG, "null argument");
    const int S = ctx->slabs.S > 1 ? ctx->slabs.S : 0;
    if (out && *n_slabs < S) return fail(nullptr, IBL_ERR_ARG, "slab buffer too small");
    if (out) std::copy(ctx->slabs.sl.begin(), ctx->slabs.sl.begin() + S, out);
    *n_slabs = S;
    return IBL_OK;
}

ibl_status ibl_save_state(ibl_ctx* ctx, void* buf, size_t* bytes) {
    if (!ctx || !bytes) return fail(ctx, IBL_ERR_ARG, "null argument");
    CKS(finalize(ctx));
    const size_t need = state_bytes(ctx);
    if (!buf) {
        *bytes = need;
        return IBL_OK;
    }
    if (*bytes < need) return fail(ctx, IBL_ERR_ARG, "state buffer too small: " + std::to_string(need) + " bytes needed");
    CKS(enter(ctx));
    const StateHeader h = state_header(ctx);
    std::memcpy(buf, &h, sizeof(h));
    size_t off = sizeof(h);
    for (const StateSection& s : state_sections(ctx)) {
        if (s.bytes) CK(cudaMemcpyAsync((char*)buf + off, s.dev, s.bytes, cudaMemcpyDeviceToHost, ctx->work));
        off += s.bytes;
    }
    CK(cudaStreamSynchronize(ctx->work));
    CKS(leave(ctx));
    *bytes = need;
    return IBL_OK;
}

ibl_status ibl_load_state(ibl_ctx* ctx, const void* buf, size_t bytes) {
    if (!ctx || !buf) return fail(ctx, IBL_ERR_ARG, "null argument");
    CKS(finalize(ctx));
    const size_t need = state_bytes(ctx);
    StateHeader h{};
    if (bytes < sizeof(h)) return fail(ctx, IBL_ERR_ARG, "state buffer too small");
    std::memcpy(&h, buf, sizeof(h));
    const StateHeader mine = state_header(ctx);
    if (std::memcmp(h.magic, mine.magic, 8) != 0 || h.version != mine.version)
        return fail(ctx, IBL_ERR_ARG, "not a state snapshot of this library version");
    if (h.storage != mine.storage || h.f_bytes != mine.f_bytes || h.n_members != mine.n_members ||
        h.n_caps != mine.n_caps || h.n_verts != mine.n_verts || bytes < need)
        return fail(ctx, IBL_ERR_ARG, "state snapshot of a different set-up (lattices, storage or capsules)");
    CKS(enter(ctx));
    size_t off = sizeof(h);
    for (const StateSection& s : state_sections(ctx)) {
        if (s.bytes) CK(cudaMemcpyAsync(s.dev, (const char*)buf + off, s.bytes, cudaMemcpyHostToDevice, ctx->work));
        off += s.bytes;
    }
    CK(launch_mirror(ctx->dev, ctx->work));   // derived from x
    ctx->t = h.t;
    CKS(sync_host_state(ctx));
    CKS(leave(ctx));
    return IBL_OK;
}

ibl_status ibl_adjoint_flow(ibl_ctx* ctx, int32_t n_steps, int32_t ckpt_every, const ibl_objective* obj,
                            double* J_out, double* grad_inlet_scale, double* grad_rj) {
    if (!ctx || !obj) return fail(ctx, IBL_ERR_ARG, "null argument");
    if (n_steps < 1 || ckpt_every < 1) return fail(ctx, IBL_ERR_ARG, "n_steps and ckpt_every must be >= 1");
    CKS(finalize(ctx));
    DevState& D = ctx->dev;
    if (D.n_members != 1 || D.n_caps != 0 || ctx->storage != IBL_STORAGE_F32)
        return fail(ctx, IBL_ERR_STATE, "the flow adjoint covers one FP32 lattice without capsules (ibl_adjoint "
                                        "differentiates a capsule objective)");
    const MemberDev& md = ctx->hmem[0];
    const size_t N = (size_t)md.N, LS = N;
    const int K = std::min(ckpt_every, n_steps);
    const int n_ck = (n_steps + K - 1) / K;
    const std::vector<StateSection> secs = state_sections(ctx);
    size_t snap_bytes = 0;
    for (const StateSection& sc : secs) snap_bytes += sc.bytes;
    // work buffers: allocated by the first call (or a call that needs more
    // checkpoints or a longer segment) and kept in the context
    auto& AC = ctx->adj;
    const size_t ck_need = (size_t)(n_ck - 1) * D.f_bytes;   // no copy when one segment covers the steps
    if (AC.kind != 0 || AC.ck_bytes < ck_need || AC.tape_steps < (size_t)K || !AC.acc) {
        cudaStreamSynchronize(ctx->work);
        free_adjoint(ctx);
        AC.kind = 0;
        auto alloc = [&](size_t bytes, void** p) -> ibl_status {
            const cudaError_t e = cudaMalloc(p, std::max<size_t>(bytes, 16));
            if (e != cudaSuccess) {
                *p = nullptr;
                return fail(ctx, IBL_ERR_OOM, "adjoint buffers: cudaMalloc of " + std::to_string(bytes) + " bytes failed");
            }
            return IBL_OK;
        };
        ibl_status ast = IBL_OK;
        if (ast == IBL_OK) ast = alloc(ck_need, (void**)&AC.ck);
        if (ast == IBL_OK) ast = alloc(snap_bytes, (void**)&AC.snap);
        if (ast == IBL_OK) ast = alloc((size_t)K * N * sizeof(float4), (void**)&AC.tape_rhou);
        if (ast == IBL_OK) ast = alloc((size_t)K * D.n_links * sizeof(float), (void**)&AC.tape_dvdq);
        if (ast == IBL_OK) ast = alloc((size_t)K * D.n_face_nodes * sizeof(float), (void**)&AC.tape_rho);
        if (ast == IBL_OK) ast = alloc(Q * LS * sizeof(float), (void**)&AC.lamA);
        if (ast == IBL_OK) ast = alloc(Q * LS * sizeof(float), (void**)&AC.lamB);
        if (ast == IBL_OK) ast = alloc(3 * sizeof(double), (void**)&AC.acc);
        if (ast != IBL_OK) { free_adjoint(ctx); return ast; }
        AC.ck_bytes = ck_need;
        AC.tape_steps = (size_t)K;
    }
    char *ck = AC.ck, *snap = AC.snap;
    float4* tape_rhou = AC.tape_rhou;
    float *tape_dvdq = AC.tape_dvdq, *tape_rho = AC.tape_rho, *lamA = AC.lamA, *lamB = AC.lamB;
    double* acc = AC.acc;   // J, dJ/ds_u, dJ/dr_j
    auto run = [&]() -> ibl_status {
        cudaStream_t s = ctx->work;
        CKS(enter(ctx));
        // solid entries of both lambda buffers start at zero (they then hold
        // only the link terms of one step at a time)
        CK(cudaMemsetAsync(lamA, 0, Q * LS * sizeof(float), s));
        CK(cudaMemsetAsync(lamB, 0, Q * LS * sizeof(float), s));
        CK(cudaMemsetAsync(acc, 0, 3 * sizeof(double), s));
        const long long t0 = ctx->t;
        // Segment work, captured once per (mode, start parity, length, adjoint
        // buffer) as a CUDA graph and replayed.  Mode 0: recompute the steps
        // from the checkpoint writing the tape, then the adjoint steps
        // backwards; mode 1: the adjoint steps only (the tape is already
        // there); mode 2: forward steps writing the tape (the last segment of
        // the forward sweep, which then needs no recompute).
        std::vector<ibl_ctx::AdjSeg>& graphs = AC.graphs;
        auto enqueue_segment = [&](int mode, int parity0, int len, float* lin0) -> ibl_status {
            if (mode != 1)
                for (int k = 0; k < len; ++k) {
                    const int parity = (parity0 + k) & 1;
                    if (mode == 2) CK(launch_step_begin(D, s));
                    CK(launch_lbm(D, parity, s, tape_rhou + (size_t)k * N));
                    CK(launch_walls(D, parity, s, tape_dvdq + (size_t)k * D.n_links,
                                    tape_rho + (size_t)k * D.n_face_nodes));
                }
            if (mode != 2) {
                float* li = lin0;
                float* lo = lin0 == lamA ? lamB : lamA;
                for (int k = len - 1; k >= 0; --k) {
                    CK(launch_adj_step(D, tape_rho + (size_t)k * D.n_face_nodes, tape_dvdq + (size_t)k * D.n_links,
                                       tape_rhou + (size_t)k * N, li, lo, LS, acc + 1, acc + 2, s));
                    std::swap(li, lo);
                }
            }
            return IBL_OK;
        };
        auto run_segment = [&](int mode, int parity0, int len, float* lin0) -> ibl_status {
            for (const ibl_ctx::AdjSeg& g : graphs)
                if (g.kind == 0 && g.mode == mode && g.parity == parity0 && g.len == len && g.lin == lin0) {
                    CK(cudaGraphLaunch(g.exec, s));
                    return IBL_OK;
                }
            cudaGraph_t gr = nullptr;
            CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
            const ibl_status est = enqueue_segment(mode, parity0, len, lin0);
            const cudaError_t e = cudaStreamEndCapture(s, &gr);
            if (est != IBL_OK) { if (gr) cudaGraphDestroy(gr); return est; }
            CK(e);
            cudaGraphExec_t ex = nullptr;
            const cudaError_t ei = cudaGraphInstantiate(&ex, gr, 0);
            cudaGraphDestroy(gr);
            CK(ei);
            graphs.push_back({0, mode, parity0, len, lin0, 0, ex});
            CK(cudaGraphLaunch(ex, s));
            return IBL_OK;
        };
        // forward sweep with a checkpoint of the populations at the start of
        // every segment but the last, which records its tape directly
        const int last0 = (n_ck - 1) * K;
        for (int k = 0; k < last0; ++k) {
            if (k % K == 0)
                CK(cudaMemcpyAsync(ck + (size_t)(k / K) * D.f_bytes, D.f, D.f_bytes, cudaMemcpyDeviceToDevice, s));
            const int parity = (int)(ctx->t & 1);
            if (ctx->use_graphs) {
                CKS(capture_graph(ctx, parity));
                CK(cudaGraphLaunch(ctx->graph[parity], s));
            } else {
                CKS(enqueue_step(ctx, parity, nullptr));
            }
            ctx->t += 1;
        }
        CKS(run_segment(2, (int)(ctx->t & 1), n_steps - last0, lamA));
        ctx->t += n_steps - last0;
        const int lo[3] = {obj->lo[0], obj->lo[1], obj->lo[2]}, hi[3] = {obj->hi[0], obj->hi[1], obj->hi[2]};
        CK(launch_adj_objective(D, (int)(ctx->t & 1), lo, hi, obj->d, lamA, LS, acc, s));
        {   // the final state, put back after the reverse sweep
            size_t off = 0;
            for (const StateSection& sc : secs) {
                if (sc.bytes) CK(cudaMemcpyAsync(snap + off, sc.dev, sc.bytes, cudaMemcpyDeviceToDevice, s));
                off += sc.bytes;
            }
        }
        float* lin = lamA;
        ibl_status sst = IBL_OK;
        for (int seg = n_ck - 1; seg >= 0 && sst == IBL_OK; --seg) {
            const int s0 = seg * K, s1 = std::min(n_steps, s0 + K);
            if (seg < n_ck - 1) {
                const cudaError_t e = cudaMemcpyAsync(D.f, ck + (size_t)seg * D.f_bytes, D.f_bytes,
                                                      cudaMemcpyDeviceToDevice, s);
                if (e != cudaSuccess) { sst = fail(ctx, IBL_ERR_CUDA, cudaGetErrorString(e)); break; }
            }
            sst = run_segment(seg < n_ck - 1 ? 0 : 1, (int)((t0 + s0) & 1), s1 - s0, lin);
            if ((s1 - s0) & 1) lin = lin == lamA ? lamB : lamA;
        }
        CKS(sst);
        {
            size_t off = 0;
            for (const StateSection& sc : secs) {
                if (sc.bytes) CK(cudaMemcpyAsync(sc.dev, snap + off, sc.bytes, cudaMemcpyDeviceToDevice, s));
                off += sc.bytes;
            }
        }
        ctx->t = t0 + n_steps;
        double h[3];
        CK(cudaMemcpyAsync(h, acc, sizeof(h), cudaMemcpyDeviceToHost, s));
        CKS(sync_host_state(ctx));
        CKS(leave(ctx));
        if (J_out) *J_out = h[0];
        if (grad_inlet_scale) *grad_inlet_scale = h[1];
        if (grad_rj) *grad_rj = h[2];
        return IBL_OK;
    };
    return run();
}

ibl_status ibl_adjoint(ibl_ctx* ctx, int32_t n_steps, int32_t ckpt_every, const double* dJ_dD_dOffset,
                       double* grad_Ca, double* grad_umax, double* grad_rj) {
    if (!ctx || !dJ_dD_dOffset) return fail(ctx, IBL_ERR_ARG, "null argument");
    if (n_steps < 1 || ckpt_every < 1) return fail(ctx, IBL_ERR_ARG, "n_steps and ckpt_every must be >= 1");
    CKS(finalize(ctx));
    DevState& D = ctx->dev;
    if (D.n_members != 1 || ctx->storage != IBL_STORAGE_F32 || D.n_caps != 1 || D.any_rigid)
        return fail(ctx, IBL_ERR_STATE, "the capsule adjoint covers one FP32 lattice holding one soft capsule "
                                        "(ibl_adjoint_flow differentiates a flow objective without capsules)");
    const MemberDev& md = ctx->hmem[0];
    const size_t N = (size_t)md.N, LS = N;
    const int nv = D.n_verts;
    const size_t nv3 = 3 * (size_t)nv;
    const int K = std::min(ckpt_every, n_steps);
    const int n_ck = (n_steps + K - 1) / K;
    const std::vector<StateSection> secs = state_sections(ctx);
    size_t snap_bytes = 0;
    for (const StateSection& sc : secs) snap_bytes += sc.bytes;
    // a checkpoint: the populations and the vertex state x, x(t - dt), v
    const size_t cap_bytes = 3 * nv3 * sizeof(double);
    const size_t ck_one = D.f_bytes + cap_bytes;
    const size_t ck_need = (size_t)(n_ck - 1) * ck_one;
    auto& AC = ctx->adj;
    if (AC.kind != 1 || AC.ck_bytes < ck_need || AC.tape_steps < (size_t)K || !AC.acc ||
        (n_ck > 1 && AC.tape2_steps < (size_t)K)) {
        cudaStreamSynchronize(ctx->work);
        free_adjoint(ctx);
        AC.kind = 1;
        auto alloc = [&](size_t bytes, void** p) -> ibl_status {
            const cudaError_t e = cudaMalloc(p, std::max<size_t>(bytes, 16));
            if (e != cudaSuccess) {
                cudaGetLastError();
                *p = nullptr;
                return fail(ctx, IBL_ERR_OOM, "adjoint buffers: cudaMalloc of " + std::to_string(bytes) + " bytes failed");
            }
            return IBL_OK;
        };
        AdjCapPtrs& c = AC.cp;
        ibl_status ast = IBL_OK;
        struct Req { size_t bytes; void** p; };
        const Req reqs[] = {
            {ck_need, (void**)&AC.ck},
            {snap_bytes, (void**)&AC.snap},
            {(size_t)K * N * sizeof(float4), (void**)&AC.tape_rhou},
            {(size_t)K * N * sizeof(float4), (void**)&AC.tape_F},
            {(size_t)K * D.n_links * sizeof(float), (void**)&AC.tape_dvdq},
            {(size_t)K * D.n_face_nodes * sizeof(float), (void**)&AC.tape_rho},
            {(size_t)K * nv3 * sizeof(double), (void**)&AC.tape_x},
            {(size_t)K * nv3 * sizeof(double), (void**)&AC.tape_v},
            {Q * LS * sizeof(float), (void**)&AC.lamA},
            {Q * LS * sizeof(float), (void**)&AC.lamB},
            {4 * sizeof(double), (void**)&AC.acc},
            {nv * sizeof(float4), (void**)&c.lx},
            {nv * sizeof(float4), (void**)&c.lxp},
            {nv * sizeof(float4), (void**)&c.lv},
            {nv * sizeof(float4), (void**)&c.lU},
            {nv * sizeof(float4), (void**)&c.lF},
            {nv * sizeof(float4), (void**)&c.ln},
            {nv * sizeof(float), (void**)&c.lA},
            {nv * sizeof(float), (void**)&c.snorm},
            {(size_t)D.n_caps * sizeof(double), (void**)&c.lV},
            {N * sizeof(float4), (void**)&c.lfib},
            {N * sizeof(float4), (void**)&c.lmac},
            {n_ck > 1 ? (size_t)K * N * sizeof(float4) : 0, (void**)&AC.tape2_rhou},
            {n_ck > 1 ? (size_t)K * N * sizeof(float4) : 0, (void**)&AC.tape2_F},
            {n_ck > 1 ? (size_t)K * D.n_links * sizeof(float) : 0, (void**)&AC.tape2_dvdq},
            {n_ck > 1 ? (size_t)K * D.n_face_nodes * sizeof(float) : 0, (void**)&AC.tape2_rho},
            {n_ck > 1 ? (size_t)K * nv3 * sizeof(double) : 0, (void**)&AC.tape2_x},
            {n_ck > 1 ? (size_t)K * nv3 * sizeof(double) : 0, (void**)&AC.tape2_v},
            {nv3 * sizeof(double), (void**)&AC.rx},
            {2 * (size_t)nv * sizeof(float4), (void**)&AC.rxm},
            {(size_t)nv * sizeof(float4), (void**)&AC.rvacc},
            {nv3 * sizeof(float), (void**)&AC.rnrm},
            {(size_t)nv * sizeof(float), (void**)&AC.rarea},
            {(size_t)D.n_caps * sizeof(CapsuleSums), (void**)&AC.rsums},
        };
        for (const Req& r : reqs)
            if (ast == IBL_OK) ast = alloc(r.bytes, r.p);
        if (ast != IBL_OK) { free_adjoint(ctx); return ast; }
        cudaError_t ce = cudaStreamCreateWithFlags(&AC.rs, cudaStreamNonBlocking);
        for (cudaEvent_t* e : {&AC.ev_rec[0], &AC.ev_rec[1], &AC.ev_rev[0], &AC.ev_rev[1], &AC.ev_fwd})
            if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(e, cudaEventDisableTiming);
        if (ce == cudaSuccess) ce = cudaMemsetAsync(AC.rvacc, 0, (size_t)nv * sizeof(float4), ctx->work);
        if (ce != cudaSuccess) {
            free_adjoint(ctx);
            return fail(ctx, IBL_ERR_CUDA, std::string("adjoint streams: ") + cudaGetErrorString(ce));
        }
        AC.ck_bytes = ck_need;
        AC.tape_steps = (size_t)K;
        AC.tape2_steps = n_ck > 1 ? (size_t)K : 0;
    }
    AdjCapPtrs cp = AC.cp;
    cp.acc_ca = AC.acc + 3;
    char *ck = AC.ck, *snap = AC.snap;
    float *lamA = AC.lamA, *lamB = AC.lamB;
    double* acc = AC.acc;   // [1] dJ/ds_u, [2] dJ/dr_j, [3] sum F_sb . lambda_F
    const MemberHost& M0 = ctx->members[0];
    const double Ca = M0.caps[0].p.Ca, u_max = M0.desc.u_max;
    cudaStream_t s = ctx->work;
    // the reverse sweep rebuilds the geometry of every step in its own
    // buffers, so that the recompute of the previous segment can run on the
    // forward buffers at the same time
    DevState Dr = D;
    Dr.x = AC.rx;
    Dr.xm = AC.rxm;
    Dr.vacc = AC.rvacc;
    Dr.nrm = AC.rnrm;
    Dr.area = AC.rarea;
    Dr.sums = AC.rsums;
    cudaStream_t rs = AC.rs;
    auto tape_of = [&](int k, int b) {
        StepTape tp;
        tp.rhou = (b ? AC.tape2_rhou : AC.tape_rhou) + (size_t)k * N;
        tp.F = (b ? AC.tape2_F : AC.tape_F) + (size_t)k * N;
        tp.dvdq = (b ? AC.tape2_dvdq : AC.tape_dvdq) + (size_t)k * D.n_links;
        tp.rho = (b ? AC.tape2_rho : AC.tape_rho) + (size_t)k * D.n_face_nodes;
        tp.x = (b ? AC.tape2_x : AC.tape_x) + (size_t)k * nv3;
        tp.v = (b ? AC.tape2_v : AC.tape_v) + (size_t)k * nv3;
        return tp;
    };
    // Segment work, captured once per (mode, start parity, length, adjoint
    // buffer, tape) as a CUDA graph: mode 1 runs the adjoint steps backwards
    // over a tape; mode 2 runs the forward steps writing the tape.
    auto enqueue_segment = [&](int mode, int parity0, int len, float* lin0, int b) -> ibl_status {
        if (mode == 2)
            for (int k = 0; k < len; ++k) {
                const StepTape tp = tape_of(k, b);
                CKS(enqueue_step(ctx, (parity0 + k) & 1, nullptr, &tp));
            }
        if (mode == 1) {
            float* li = lin0;
            float* lo = lin0 == lamA ? lamB : lamA;
            for (int k = len - 1; k >= 0; --k) {
                const StepTape tp = tape_of(k, b);
                CK(launch_adj_step(D, tp.rho, tp.dvdq, tp.rhou, li, lo, LS, acc + 1, acc + 2, s, tp.F, cp.lfib));
                CK(cudaMemcpyAsync(Dr.x, tp.x, nv3 * sizeof(double), cudaMemcpyDeviceToDevice, s));
                CK(launch_mirror(Dr, s));
                CK(launch_adj_geometry(Dr, cp.lV, cp.snorm, s));
                CK(launch_adj_capsules(Dr, cp, tp.rhou, tp.F, tp.v, lo, LS, s));
                std::swap(li, lo);
            }
        }
        return IBL_OK;
    };
    // launch on `on` (a graph is captured on the work stream the first time,
    // with both streams idle)
    auto run_segment = [&](int mode, int parity0, int len, float* lin0, int b, cudaStream_t on) -> ibl_status {
        for (const ibl_ctx::AdjSeg& g : AC.graphs)
            if (g.kind == 1 && g.mode == mode && g.parity == parity0 && g.len == len && g.lin == lin0 && g.tb == b) {
                CK(cudaGraphLaunch(g.exec, on));
                return IBL_OK;
            }
        CK(cudaStreamSynchronize(s));
        CK(cudaStreamSynchronize(rs));
        cudaGraph_t gr = nullptr;
        CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        const ibl_status est = enqueue_segment(mode, parity0, len, lin0, b);
        const cudaError_t e = cudaStreamEndCapture(s, &gr);
        if (est != IBL_OK) { if (gr) cudaGraphDestroy(gr); return est; }
        CK(e);
        cudaGraphExec_t ex = nullptr;
        const cudaError_t ei = cudaGraphInstantiate(&ex, gr, 0);
        cudaGraphDestroy(gr);
        CK(ei);
        AC.graphs.push_back({1, mode, parity0, len, lin0, b, ex});
        CK(cudaGraphLaunch(ex, on));
        return IBL_OK;
    };
    auto copy_caps = [&](char* base, bool save) -> ibl_status {
        double* dst[3] = {D.x, D.x_prev, D.vel};
        for (int i = 0; i < 3; ++i) {
            char* h = base + D.f_bytes + i * nv3 * sizeof(double);
            if (save) CK(cudaMemcpyAsync(h, dst[i], nv3 * sizeof(double), cudaMemcpyDeviceToDevice, s));
            else CK(cudaMemcpyAsync(dst[i], h, nv3 * sizeof(double), cudaMemcpyDeviceToDevice, s));
        }
        if (save) CK(cudaMemcpyAsync(base, D.f, D.f_bytes, cudaMemcpyDeviceToDevice, s));
        else {
            CK(cudaMemcpyAsync(D.f, base, D.f_bytes, cudaMemcpyDeviceToDevice, s));
            CK(launch_mirror(D, s));
        }
        return IBL_OK;
    };
    CKS(enter(ctx));
    CK(cudaMemsetAsync(lamA, 0, Q * LS * sizeof(float), s));
    CK(cudaMemsetAsync(lamB, 0, Q * LS * sizeof(float), s));
    CK(cudaMemsetAsync(acc, 0, 4 * sizeof(double), s));
    CK(cudaMemsetAsync(cp.lmac, 0, N * sizeof(float4), s));
    CK(cudaMemsetAsync(cp.lfib, 0, N * sizeof(float4), s));
    const long long t0 = ctx->t;
    // forward sweep: a checkpoint at the start of every segment but the last,
    // whose tape is recorded directly
    const int last0 = (n_ck - 1) * K;
    for (int k = 0; k < last0; ++k) {
        if (k % K == 0) CKS(copy_caps(ck + (size_t)(k / K) * ck_one, true));
        const int parity = (int)(ctx->t & 1);
        CKS(capture_graph(ctx, parity));
        CK(cudaGraphLaunch(ctx->graph[parity], s));
        ctx->t += 1;
    }
    const int L = n_ck - 1;
    CKS(run_segment(2, (int)(ctx->t & 1), n_steps - last0, lamA, L & 1, s));
    ctx->t += n_steps - last0;
    // terminal condition: lambda_x = dJ/dx at the last step (FP64, host)
    std::vector<double> XT(nv3), G(nv3);
    CK(cudaMemcpyAsync(XT.data(), D.x, nv3 * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    const std::vector<int>& tris = M0.caps[0].tris;
    capsule_objective_grad(XT.data(), nv, tris.data(), (int)tris.size() / 3, dJ_dD_dOffset[0], dJ_dD_dOffset[1],
                           G.data());
    {
        std::vector<float4> L4(nv);
        for (int v = 0; v < nv; ++v)
            L4[v] = make_float4((float)G[3 * v], (float)G[3 * v + 1], (float)G[3 * v + 2], 0.f);
        CK(cudaMemcpyAsync(cp.lx, L4.data(), nv * sizeof(float4), cudaMemcpyHostToDevice, s));
        CK(cudaMemsetAsync(cp.lxp, 0, nv * sizeof(float4), s));
        CK(cudaMemsetAsync(cp.lv, 0, nv * sizeof(float4), s));
        CK(cudaStreamSynchronize(s));
    }
    {   // the final state, put back after the reverse sweep
        size_t off = 0;
        for (const StateSection& sc : secs) {
            if (sc.bytes) CK(cudaMemcpyAsync(snap + off, sc.dev, sc.bytes, cudaMemcpyDeviceToDevice, s));
            off += sc.bytes;
        }
    }
    // reverse sweep on stream rs, segment by segment from the last; the
    // recompute of segment seg - 1 (on the work stream, into the other tape)
    // runs beside the reverse of segment seg
    CK(cudaEventRecord(AC.ev_fwd, s));
    float* lin = lamA;
    for (int seg = L; seg >= 0; --seg) {
        if (seg >= 1) {
            const int p = seg - 1, b = p & 1;
            if (seg + 1 <= L) CK(cudaStreamWaitEvent(s, AC.ev_rev[b], 0));   // tape b free again
            CKS(copy_caps(ck + (size_t)p * ck_one, false));
            CKS(run_segment(2, (int)((t0 + (long long)p * K) & 1), K, lamA, b, s));
            CK(cudaEventRecord(AC.ev_rec[b], s));
        }
        const int s0 = seg * K, s1 = std::min(n_steps, s0 + K), b = seg & 1;
        CK(cudaStreamWaitEvent(rs, seg == L ? AC.ev_fwd : AC.ev_rec[b], 0));
        CKS(run_segment(1, (int)((t0 + s0) & 1), s1 - s0, lin, b, rs));
        CK(cudaEventRecord(AC.ev_rev[b], rs));
        if ((s1 - s0) & 1) lin = lin == lamA ? lamB : lamA;
    }
    CK(cudaEventRecord(AC.ev_fwd, rs));
    CK(cudaStreamWaitEvent(s, AC.ev_fwd, 0));
    {
        size_t off = 0;
        for (const StateSection& sc : secs) {
            if (sc.bytes) CK(cudaMemcpyAsync(sc.dev, snap + off, sc.bytes, cudaMemcpyDeviceToDevice, s));
            off += sc.bytes;
        }
        CK(launch_mirror(D, s));
    }
    ctx->t = t0 + n_steps;
    double h[4];
    CK(cudaMemcpyAsync(h, acc, sizeof(h), cudaMemcpyDeviceToHost, s));
    CKS(sync_host_state(ctx));
    CKS(leave(ctx));
    if (grad_Ca) *grad_Ca = -h[3] / Ca;
    if (grad_umax) *grad_umax = u_max != 0.0 ? h[1] / u_max : 0.0;
    if (grad_rj) *grad_rj = h[2];
    uint32_t any = 0;
    for (uint32_t st : ctx->h_status) any |= st;
    if (any & ST_NONFINITE) return fail(ctx, IBL_ERR_NONFINITE, "a capsule vertex became non-finite");
    if (any & ST_DAMAGED) return fail(ctx, IBL_ERR_DAMAGED, "a capsule edge reached twice its rest length");
    return IBL_OK;
}

ibl_status ibl_read_fields_noalloc(ibl_ctx* ctx, int32_t member, float* rho, float* u) {
    if (!ctx) return fail(nullptr, IBL_ERR_ARG, "null context");
    if (!rho && !u) return fail(ctx, IBL_ERR_ARG, "null outputs");
    if (member < 0 || member >= (int)ctx->members.size()) return fail(ctx, IBL_ERR_ARG, "member out of range");
    if (ctx->members[member].whole_view)
        return fail(ctx, IBL_ERR_ARG, "the whole-lattice member of a slab context holds no populations");
    const ibl_lattice_desc& dsc = ctx->members[member].desc;
    const size_t Nu = (size_t)dsc.nx * dsc.ny * dsc.nz;
    if (Nu > (size_t)IBL_NOALLOC_MAX_NODES)
        return fail(ctx, IBL_ERR_ARG, "lattice of " + std::to_string(Nu) + " nodes exceeds the static read array (" +
                                          std::to_string(IBL_NOALLOC_MAX_NODES) +
                                          " nodes, IBL_NOALLOC_MAX_NODES); use ibl_member_read_fields");
    if (!ctx->finalized)
        return fail(ctx, IBL_ERR_STATE, "no device state yet (its set-up allocates): step, initialise or read first");
    int dev = -1;
    CK(cudaGetDevice(&dev));
    if (dev != ctx->device || !ctx->noalloc)
        return fail(ctx, IBL_ERR_STATE, "the context's device (" + std::to_string(ctx->device) +
                                            ") must be current (device " + std::to_string(dev) + " is)");
    float* scratch = ctx->noalloc;
    float* dr = rho ? scratch : nullptr;
    float* du = u ? scratch + IBL_NOALLOC_MAX_NODES : nullptr;
    const int cnt = ctx->h_counters[member];
    CKS(enter(ctx));
    CK(launch_read(ctx->dev, member, cnt & 1, dr, du, nullptr, ctx->work));
    if (rho) CK(cudaMemcpyAsync(rho, dr, sizeof(float) * Nu, cudaMemcpyDeviceToHost, ctx->work));
    if (u) CK(cudaMemcpyAsync(u, du, sizeof(float) * 3 * Nu, cudaMemcpyDeviceToHost, ctx->work));
    CK(cudaStreamSynchronize(ctx->work));
    CKS(leave(ctx));
    return IBL_OK;
}

int32_t ibl_num_members(const ibl_ctx* ctx) { return ctx ? (int32_t)ctx->members.size() : 0; }

ibl_status ibl_member_read_fields(ibl_ctx* ctx, int32_t member, float* rho, float* u, int32_t on_device) {
    if (!ctx) return fail(nullptr, IBL_ERR_ARG, "null context");
    return read_fields_member(ctx, member, rho, u, nullptr, on_device);
}

ibl_status ibl_member_read_populations(ibl_ctx* ctx, int32_t member, float* g, int32_t on_device) {
    if (!ctx) return fail(nullptr, IBL_ERR_ARG, "null context");
    if (!g) return fail(ctx, IBL_ERR_ARG, "null output");
    return read_fields_member(ctx, member, nullptr, nullptr, g, on_device);
}

ibl_status ibl_member_read_capsule(ibl_ctx* ctx, int32_t member, int32_t id, ibl_capsule_stats* stats,
                                   double* verts_out) {
    if (!ctx) return fail(nullptr, IBL_ERR_ARG, "null context");
    return read_capsule_member(ctx, member, id, stats, verts_out);
}

ibl_status ibl_member_steps(const ibl_ctx* ctx, int32_t member, int32_t* steps_done) {
    if (!ctx || !steps_done) return fail(nullptr, IBL_ERR_ARG, "null argument");
    if (member < 0 || member >= (int)ctx->members.size()) return fail(nullptr, IBL_ERR_ARG, "member out of range");
    *steps_done = ctx->finalized ? ctx->h_counters[member] : 0;
    return IBL_OK;
}

ibl_status ibl_set_launch(ibl_ctx* ctx, int32_t threads, int32_t blocks_per_sm) {
    if (!ctx) return fail(nullptr, IBL_ERR_ARG, "null context");
    if (threads < 32 || threads > lbm_max_threads() || threads % 32 || blocks_per_sm < 0 || blocks_per_sm > 64)
        return fail(ctx, IBL_ERR_ARG, "threads must be a multiple of 32 in [32, " + std::to_string(lbm_max_threads()) +
                                          "], blocks_per_sm in [0, 64]");
    ctx->threads = threads;
    ctx->blocks_per_sm = blocks_per_sm;
    if (ctx->finalized) {
        CK(cudaStreamSynchronize(ctx->work));
        layout_tiles(ctx);
        CKS(upload(ctx, ctx->dev.mem, ctx->hmem));
        CK(cudaStreamSynchronize(ctx->work));
        drop_graphs(ctx);
    }
    return IBL_OK;
}

ibl_status ibl_set_lattice_path(ibl_ctx* ctx, int32_t staged) {
    if (!ctx) return fail(nullptr, IBL_ERR_ARG, "null context");
    if (staged != 0 && staged != 1) return fail(ctx, IBL_ERR_ARG, "staged must be 0 or 1");
    ctx->lattice_path = staged;
    if (ctx->finalized) {
        CK(cudaStreamSynchronize(ctx->work));
        DevState& D = ctx->dev;
        if (staged && !D.chunks && ctx->members.size() == 1 && D.n_groups > 0) {
            // the chunks come from the interior work list on the device
            std::vector<uint32_t> nodes((size_t)D.n_groups * 32);
            CK(cudaMemcpy(nodes.data(), D.nodes, nodes.size() * sizeof(uint32_t), cudaMemcpyDeviceToHost));
            CKS(build_chunks(ctx, nodes));
            CK(cudaStreamSynchronize(ctx->work));
            CKS(prepare_staged(ctx));
        }
        D.lattice_path = staged;
        drop_graphs(ctx);
    }
    return IBL_OK;
}

int32_t ibl_lattice_path(const ibl_ctx* ctx) {
    if (!ctx || !ctx->finalized) return -1;
    const DevState& D = ctx->dev;
    return (D.lattice_path == 1 && D.chunks && D.bulk_blocks_per_sm > 0) ? 1 : 0;
}

ibl_status ibl_autotune(ibl_ctx* ctx, int32_t steps, int32_t* threads_out, int32_t* blocks_per_sm_out,
                        double* ms_out) {
    if (!ctx) return fail(nullptr, IBL_ERR_ARG, "null context");
    if (steps < 1) return fail(ctx, IBL_ERR_ARG, "steps must be >= 1");
    CKS(finalize(ctx));
    // device-side snapshot of the dynamic state, restored after every trial
    const std::vector<StateSection> secs = state_sections(ctx);
    size_t total = 0;
    for (const StateSection& sc : secs) total += sc.bytes;
    char* snap = nullptr;
    CK(cudaMalloc((void**)&snap, std::max<size_t>(total, 1)));
    auto copy_state = [&](bool save) -> ibl_status {
        size_t off = 0;
        for (const StateSection& sc : secs) {
            if (sc.bytes) {
                const cudaError_t e = save ? cudaMemcpyAsync(snap + off, sc.dev, sc.bytes, cudaMemcpyDeviceToDevice, ctx->work)
                                           : cudaMemcpyAsync(sc.dev, snap + off, sc.bytes, cudaMemcpyDeviceToDevice, ctx->work);
                if (e != cudaSuccess) return fail(ctx, IBL_ERR_CUDA, std::string("state copy: ") + cudaGetErrorString(e));
            }
            off += sc.bytes;
        }
        if (!save) {
            const cudaError_t e = launch_mirror(ctx->dev, ctx->work);   // derived from x
            if (e != cudaSuccess) return fail(ctx, IBL_ERR_CUDA, std::string("mirror: ") + cudaGetErrorString(e));
        }
        return IBL_OK;
    };
    const long long t0 = ctx->t;
    const bool timing0 = ctx->timing;
    const int thr0 = ctx->threads, bps0 = ctx->blocks_per_sm;
    ibl_status st = enter(ctx);
    if (st == IBL_OK) st = copy_state(true);
    int best_t = thr0, best_b = bps0;
    double best = 1e300;
    const int cand_t[3] = {32, 64, 128};
    const int cand_b[6] = {0, 1, 2, 4, 8, 16};
    ctx->timing = true;
    for (int it = 0; it < 3 && st == IBL_OK; ++it) {
        if (cand_t[it] > lbm_max_threads()) continue;
        for (int ib = 0; ib < 6 && st == IBL_OK; ++ib) {
            if (cand_b[ib] * cand_t[it] > 2048) continue;
            st = ibl_set_launch(ctx, cand_t[it], cand_b[ib]);
            if (st == IBL_OK) st = ibl_step(ctx, steps, nullptr);
            if (st == IBL_ERR_DAMAGED || st == IBL_ERR_NONFINITE) st = IBL_OK;   // the state is restored below
            const double ms = ctx->ktime[0] / steps;
            if (st == IBL_OK && ms < best) { best = ms; best_t = cand_t[it]; best_b = cand_b[ib]; }
            if (st == IBL_OK) st = copy_state(false);
            ctx->t = t0;
            if (st == IBL_OK) st = sync_host_state(ctx);
        }
    }
    ctx->timing = timing0;
    const ibl_status st_launch = ibl_set_launch(ctx, st == IBL_OK ? best_t : thr0, st == IBL_OK ? best_b : bps0);
    cudaStreamSynchronize(ctx->work);
    cudaFree(snap);
    if (st != IBL_OK) return st;
    CKS(st_launch);
    CKS(leave(ctx));
    if (threads_out) *threads_out = best_t;
    if (blocks_per_sm_out) *blocks_per_sm_out = best_b;
    if (ms_out) *ms_out = best;
    return IBL_OK;
}

ibl_status ibl_kernels_per_step(ibl_ctx* ctx, int32_t* n) {
    if (!ctx || !n) return fail(ctx, IBL_ERR_ARG, "null argument");
    CKS(finalize(ctx));
    CKS(capture_graph(ctx, 1));
    *n = ctx->graph_kernels[1];
    return IBL_OK;
}

ibl_status ibl_enable_timing(ibl_ctx* ctx, int32_t on) {
    if (!ctx) return fail(nullptr, IBL_ERR_ARG, "null context");
    ctx->timing = on != 0;
    return IBL_OK;
}

ibl_status ibl_kernel_times(ibl_ctx* ctx, double* out4) {
    if (!ctx || !out4) return fail(ctx, IBL_ERR_ARG, "null argument");
    for (int i = 0; i < 4; ++i) out4[i] = ctx->ktime[i];
    return IBL_OK;
}

ibl_status ibl_voxelise_markers(const double* verts, int32_t n_verts, const int32_t* tris, int32_t n_tris,
                                int32_t nx, int32_t ny, int32_t nz, const int32_t* periodic,
                                const uint8_t* tag_in, uint8_t* tag_out, uint32_t* link_node,
                                uint32_t* link_dir, float* link_q, int64_t* n_links, void* cuda_stream) {
    std::string msg;
    const int r = ibl::voxelise_markers(verts, n_verts, tris, n_tris, nx, ny, nz, periodic, tag_in, tag_out,
                                        link_node, link_dir, link_q, n_links, (cudaStream_t)cuda_stream, msg);
    if (r == 0) return IBL_OK;
    return fail(nullptr, r == -1 ? IBL_ERR_ARG : IBL_ERR_CUDA, msg);
}

const char* ibl_last_error(const ibl_ctx* ctx) { return ctx ? ctx->err.c_str() : g_last_error.c_str(); }

void ibl_destroy(ibl_ctx* ctx) {
    if (!ctx) return;
    if (ctx->work) cudaStreamSynchronize(ctx->work);
    drop_graphs(ctx);
    free_adjoint(ctx);
    for (void* p : ctx->allocs) cudaFree(p);
    if (ctx->stage) cudaFree(ctx->stage);
    if (ctx->ev_in) cudaEventDestroy(ctx->ev_in);
    if (ctx->ev_out) cudaEventDestroy(ctx->ev_out);
    if (ctx->work2) cudaStreamSynchronize(ctx->work2);
    if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
    if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
    if (ctx->ev_ib) cudaEventDestroy(ctx->ev_ib);
    if (ctx->work3) cudaStreamSynchronize(ctx->work3);
    if (ctx->ev_shell) cudaEventDestroy(ctx->ev_shell);
    if (ctx->ev_probes) cudaEventDestroy(ctx->ev_probes);
    if (ctx->work3) cudaStreamDestroy(ctx->work3);
    if (ctx->work2) cudaStreamDestroy(ctx->work2);
    if (ctx->work) cudaStreamDestroy(ctx->work);
    delete ctx;
}

}  // extern "C"
