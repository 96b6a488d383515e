// Device helpers of the immersed-boundary kernels and of their adjoint:
// shared constants, small vector helpers, the two-float position mirror,
// the MLS stencil (tensor-product weights and the closed-form inverse of the
// moment matrix) built by groups of GL lanes, the probe-record force and the
// force accumulation.
#pragma once

#include "lbm_device.cuh"

namespace ibl {

constexpr float SUPPORT_SIDE = 2.6f;   // 2 r_w (Section "No-slip conditions for moving immersed boundaries")
constexpr float ALPHA = 0.3f;          // Eq. intKernel
constexpr unsigned FULL = 0xffffffffu;
constexpr uint32_t STOP = ST_DAMAGED | ST_NONFINITE;

struct f3 { float x, y, z; };
__device__ __forceinline__ f3 sub(f3 a, f3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ f3 crs(f3 a, f3 b) { return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x}; }
__device__ __forceinline__ float dot3(f3 a, f3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ f3 scl(f3 a, float s) { return {a.x * s, a.y * s, a.z * s}; }

// Two-float mirror of the FP64 vertex positions, 32 bytes per vertex:
// (hi, 0) then (lo, 0) with hi = fl32(x) and lo = fl32(x - hi) (x - hi is
// exact).  The difference of two positions taken as (hi_a - hi_b) +
// (lo_a - lo_b) in FP32 is the FP64 difference rounded to FP32 within an ulp,
// with no FP64 arithmetic (GB300's FP64 pipe is narrow).  Written with x by
// the update kernels, and by k_mirror after x is set from the host.
__device__ __forceinline__ void mirror_put(float4* __restrict__ xm, int v, double X, double Y, double Z) {
    const float hx = (float)X, hy = (float)Y, hz = (float)Z;
    xm[2 * v] = make_float4(hx, hy, hz, 0.f);
    xm[2 * v + 1] = make_float4((float)(X - (double)hx), (float)(Y - (double)hy), (float)(Z - (double)hz), 0.f);
}

// x_a - x_b
__device__ __forceinline__ f3 mirror_diff(const float4* __restrict__ xm, int a, int b) {
    const float4 ha = xm[2 * a], la = xm[2 * a + 1], hb = xm[2 * b], lb = xm[2 * b + 1];
    return {(ha.x - hb.x) + (la.x - lb.x), (ha.y - hb.y) + (la.y - lb.y), (ha.z - hb.z) + (la.z - lb.z)};
}

// Eq. intKernel with r normalised by the support side.
__device__ __forceinline__ double block_sum_d(double v, double* red) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x < 32) {
        t = (lane < (int)(blockDim.x >> 5)) ? red[lane] : 0.0;
#pragma unroll
        for (int o = 16; o; o >>= 1) t += __shfl_xor_sync(FULL, t, o);
    }
    return t;   // valid in thread 0
}

// Moments (rho, u* = sum g e / rho) of the current populations at the fluid
// nodes that a marker or probe stencil can reach.  A marker's support lies
// within 1.5 dx of it per axis (the 3x3x3 block around its nearest node); a
// probe sits 1.2 dx off its vertex along the unit normal, so its support lies
// within 1.2 + 1.5 = 2.7 dx of the vertex per axis and within 1.2 + 1.5 sqrt 3
// < 3.8 dx of it in distance.  Per axis every support coordinate lies in
// [floor(min) - 2, floor(max) + 3], which is the vertex box
// [floor(min), floor(max) + 1] grown by SHELL_MARGIN = 2.  Within the box, a
// node farther than sqrt(r2_hi) + 3.8 from the step's reference point rc, or
// nearer than sqrt(r2_lo) - 3.8, is within 3.8 of no vertex and is skipped
// (a 0.05 slack covers the FP32 distances and square roots).  The IB kernels then read one
// float4 per support node instead of 19 scattered populations.  Overlapping
// boxes write identical values.
constexpr int SHELL_MARGIN = 2;
constexpr float SHELL_REACH = 3.85f;
constexpr int SHELL_BLOCKS = 32;   // blocks per capsule

// Offsets (dx, dy, dz) of support node k = (dx+1) + 3 (dy+1) + 9 (dz+1) of
// the 3x3x3 MLS block, packed two bits per node, so that a run-time k costs a
// shift and a mask instead of divisions.
__device__ __forceinline__ int sdx(int k) { return (int)((0x24924924924924ull >> (2 * k)) & 3ull) - 1; }
__device__ __forceinline__ int sdy(int k) { return (int)((0x2a540a9502a540ull >> (2 * k)) & 3ull) - 1; }
__device__ __forceinline__ int sdz(int k) { return (int)((0x2aaaa555540000ull >> (2 * k)) & 3ull) - 1; }

// Support node (cx, cy, cz) of a point: wrapped on a periodic axis, clamped
// to the box on the others (a point off the box takes the state of the
// nearest box node, Reading M4).
__device__ __forceinline__ int support_index(const MemberDev& d, int cx, int cy, int cz) {
    if (d.per & 1) cx = ((cx % d.nx) + d.nx) % d.nx; else cx = min(max(cx, 0), d.nx - 1);
    if (d.per & 2) cy = ((cy % d.ny) + d.ny) % d.ny; else cy = min(max(cy, 0), d.ny - 1);
    if (d.per & 4) cz = ((cz % d.nz) + d.nz) % d.nz; else cz = min(max(cz, 0), d.nz - 1);
    return (cx + d.px) + d.NX * ((cy + d.py) + d.NY * (cz + d.pz));
}

// ---------------------------------------------------------------------------
// IB marker and probe stencils, four lanes per stencil, all on the fluid
// solution at t (moments of the current populations from the shell pass):
//  s = 0: Eq. uLag on u*, F_l = (U_b - U_l)/dt, Eq. bodyforce spreading with
//         c_l = A_l into the dense f_ib field (float atomics; the shell pass
//         flags the band's fluid nodes); u_v,0 = U_l (the tentative velocity of Eq. verletPos); the
//         volume penalty k_v (1 - V/V0) A (Eq. volFor, restoring sign) of soft
//         capsules (0 for rigid ones);
//  s = 1, 2: the probe at x +- 1.2 n: p = rho/3 and tau = rho nu (grad u +
//         grad u^T) from the MLS fit (Eqs. hydroForP, hydroForNu), stored for
//         the update kernels, which add F_p + F_tau.
// Each lane gathers its support nodes' moments at once (at most GS loads in
// flight), so that their latencies overlap.
// ---------------------------------------------------------------------------
constexpr int PROBE_STRIDE = 8;   // floats per probe record: p, tau xx yy zz xy xz yz, pad
static_assert(PROBE_STRIDE == 8, "hydro_force reads each probe record as two float4");

constexpr bool PROBE_FAST32 = true;   // (template argument kept by the callers; the closed form needs no FP64 redo)
#ifndef IB_MARKER_THREADS
#define IB_MARKER_THREADS 128
#endif
#ifndef IB_MARKER_MIN_BLOCKS
#define IB_MARKER_MIN_BLOCKS 8
#endif
#ifndef IB_PROBE_THREADS
#define IB_PROBE_THREADS 128
#endif
#ifndef IB_PROBE_MIN_BLOCKS
#define IB_PROBE_MIN_BLOCKS 8
#endif
constexpr bool MARKER_FAST32 = true;

// The stencils run on groups of GL = 4 consecutive lanes: support node k of
// a point belongs to lane k % 4 (slot k / 4), so each lane gathers at most 7
// nodes, the per-axis weights and the interpolated sums are combined by
// shuffles within the group, and every lane of the group holds the same rows.  A
// stencil's latency chain is a quarter of the one-lane form and its registers
// hold 7 weights instead of 27.
#ifndef IB_GROUP_LANES
#define IB_GROUP_LANES 4
#endif
constexpr int GL = IB_GROUP_LANES;      // lanes per stencil (a power of two, at most 32)
constexpr int GS = (27 + GL - 1) / GL;  // support nodes per lane
static_assert(GL >= 4 && GL <= 32 && (GL & (GL - 1)) == 0, "a stencil group needs a lane per axis");

// MLS operator of one point, held by the GL lanes of its group: weights W_k of
// this lane's support nodes (Eq. intKernel) and the first ROWS rows of A^{-1}
// (Eq. l2norm, basis [1, x-X, y-Y, z-Z]; A is symmetric, so row j is
// A^{-1} e_j), the same in every lane of the group.
struct MlsG {
    int bx, by, bz;
    int base;               // padded index of the base node when the block is interior, else -1
    float ox, oy, oz;       // base node minus point
    float W[GS];            // weights of this lane's support nodes (k = lane + 4 slot)
    float inv[4][4];
};

// (h, l) is the point's coordinate along axis min(r, 2): lanes 0, 1, 2 of a
// group each take the nearest-node step of one axis and the group exchanges
// the results.
//
// Every point of the 3x3x3 block takes part in the fit (Reading M4: a solid
// one with the wall's state, one off the box with the nearest box node's), and
// W = exp(-|x_k - X|^2 / (2.6 alpha)^2) (every node of the block lies within
// r <= 1) is the product of one factor per axis.  The moment matrix of the
// linear basis is then
//     A = S [[1, m_x, m_y, m_z], [m_x, m_x^2 + v_x, m_x m_y, m_x m_z], ...]
// with, per axis a, s0 = sum_j w_a(j), s1 = sum_j w_a(j) r_j and
// s2 = sum_j w_a(j) r_j^2 over the offsets r_j = o_a - 1, o_a, o_a + 1 of the
// three nodes, m_a = s1 / s0, v_a = s2 / s0 - m_a^2 and S = s0_x s0_y s0_z.
// In the basis centred on m, A is diagonal, which gives the rows of A^{-1}
// below: the same operator as the general 4x4 solve of the oracle, in a few
// operations per point and with no small pivot.  Lane a (< 3) evaluates the
// three factors of axis a; the group shares them.
// With MAC the moments of every support node of the lane are gathered at once
// into q from the moments array of the step, where a solid node holds
// (-1, 0, 0, 0): the wall's rho negated, so that the spreading can skip it
// without a tag gather.
// The sum a + b of two floats as the unevaluated pair (p, e), p = fl(a + b)
// and e its rounding error, exactly (Knuth's TwoSum).
__device__ __forceinline__ void two_sum(float a, float b, float& p, float& e) {
    p = __fadd_rn(a, b);
    const float z = __fsub_rn(p, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(p, z)), __fsub_rn(b, z));
}

// The nearest node b = floor(x + 1/2) of a coordinate given as the
// unevaluated float sum x = h + l with |l| <= ulp(h) (the two-float mirror of
// an FP64 position), exactly as the FP64 floor, and the offset b - x rounded
// once: h + 1/2 is exact for |h| < 2^22; only when it is an integer does the
// sign of l decide; b - h is exact (Sterbenz).  No FP64 arithmetic (GB300's
// FP64 pipe is narrow).
__device__ __forceinline__ void nearest_of(float h, float l, int& bi, float& o) {
    const float t = __fadd_rn(h, 0.5f);
    float b = floorf(t);
    if (t == b && l < 0.f) b -= 1.f;
    bi = (int)b;
    o = __fsub_rn(__fsub_rn(b, h), l);
}

// (h, l) of an FP64 coordinate, as the mirror holds it (mirror_put)
__device__ __forceinline__ void split_of(double x, float& h, float& l) {
    h = (float)x;
    l = (float)(x - (double)h);
}

// A probe point x + s n along one axis (s = +-1.2, Section "No-slip
// conditions ..."), from the mirror (h, l) of x: the pair of h + (l + s n).
__device__ __forceinline__ void probe_of(float h, float l, float sn, float& ph, float& pl) {
    two_sum(h, __fadd_rn(l, sn), ph, pl);
}

template <int ROWS, bool MAC>
__device__ __forceinline__ void mls_build_impl(const MemberDev& d, const void* src, float h, float l, int r,
                                               unsigned mask, MlsG& M, float4 (&q)[GS]) {
    int bi;
    float o;
    nearest_of(h, l, bi, o);
    M.bx = __shfl_sync(mask, bi, 0, GL); M.by = __shfl_sync(mask, bi, 1, GL); M.bz = __shfl_sync(mask, bi, 2, GL);
    M.ox = __shfl_sync(mask, o, 0, GL); M.oy = __shfl_sync(mask, o, 1, GL); M.oz = __shfl_sync(mask, o, 2, GL);
    const bool interior = M.bx >= 1 && M.bx <= d.nx - 2 && M.by >= 1 && M.by <= d.ny - 2 && M.bz >= 1 &&
                          M.bz <= d.nz - 2;
    M.base = interior ? (M.bx + d.px) + d.NX * ((M.by + d.py) + d.NY * (M.bz + d.pz)) : -1;
    // this lane's axis factors exp(-r^2 / (2.6 alpha)^2) at r = o - 1, o, o + 1
    constexpr float L2 = 1.f / (SUPPORT_SIDE * ALPHA * SUPPORT_SIDE * ALPHA);
    const float om = o - 1.f, op = o + 1.f;
    const float wm = expf(-om * om * L2), w0 = expf(-o * o * L2), wp = expf(-op * op * L2);
    float fa[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        fa[a][0] = __shfl_sync(mask, wm, a, GL);
        fa[a][1] = __shfl_sync(mask, w0, a, GL);
        fa[a][2] = __shfl_sync(mask, wp, a, GL);
    }
    const float oa[3] = {M.ox, M.oy, M.oz};
    float m1[3], iv[3], S = 1.f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float r0 = oa[a] - 1.f, r1 = oa[a], r2 = oa[a] + 1.f;
        const float s0 = fa[a][0] + fa[a][1] + fa[a][2];
        const float s1 = fa[a][0] * r0 + fa[a][1] * r1 + fa[a][2] * r2;
        const float s2 = fa[a][0] * r0 * r0 + fa[a][1] * r1 * r1 + fa[a][2] * r2 * r2;
        const float is0 = 1.f / s0;
        m1[a] = s1 * is0;
        iv[a] = 1.f / (s2 * is0 - m1[a] * m1[a]);
        S *= s0;
    }
    const float iS = 1.f / S;
    M.inv[0][0] = (1.f + m1[0] * m1[0] * iv[0] + m1[1] * m1[1] * iv[1] + m1[2] * m1[2] * iv[2]) * iS;
#pragma unroll
    for (int a = 0; a < 3; ++a) M.inv[0][1 + a] = -m1[a] * iv[a] * iS;
    if (ROWS > 1) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            M.inv[1 + a][0] = -m1[a] * iv[a] * iS;
#pragma unroll
            for (int c = 0; c < 3; ++c) M.inv[1 + a][1 + c] = c == a ? iv[a] * iS : 0.f;
        }
    }
#pragma unroll
    for (int j = 0; j < GS; ++j) {
        const int k = r + GL * j;
        q[j] = make_float4(0.f, 0.f, 0.f, 0.f);
        M.W[j] = 0.f;
        if (k < 27) {
            const int dx = sdx(k), dy = sdy(k), dz = sdz(k);
            // register selects (the lane's node offsets are not compile-time)
            const float wx = dx < 0 ? fa[0][0] : (dx == 0 ? fa[0][1] : fa[0][2]);
            const float wy = dy < 0 ? fa[1][0] : (dy == 0 ? fa[1][1] : fa[1][2]);
            const float wz = dz < 0 ? fa[2][0] : (dz == 0 ? fa[2][1] : fa[2][2]);
            M.W[j] = wx * wy * wz;
            if (MAC) {
                const int node = interior ? M.base + dx + d.NX * (dy + d.NY * dz)
                                          : support_index(d, M.bx + dx, M.by + dy, M.bz + dz);
                q[j] = static_cast<const float4*>(src)[d.node_off + node];
            }
        }
    }
}

// the lane's coordinate along axis min(r, 2) as the pair (h, l)
template <int ROWS, bool FAST32>
__device__ __forceinline__ void mls_build_g(const MemberDev& d, const uint8_t* __restrict__ tag, float h, float l,
                                            int r, unsigned mask, MlsG& M) {
    float4 q[GS];
    mls_build_impl<ROWS, false>(d, tag, h, l, r, mask, M, q);
}

template <int ROWS, bool FAST32>
__device__ __forceinline__ void mls_build_g(const MemberDev& d, const float4* __restrict__ macro, float h, float l,
                                            int r, unsigned mask, MlsG& M, float4 (&q)[GS]) {
    mls_build_impl<ROWS, true>(d, macro, h, l, r, mask, M, q);
}

__device__ __forceinline__ float mls_row_g(const MlsG& M, int row, int j, int k) {
    const float rx = M.ox + sdx(k), ry = M.oy + sdy(k), rz = M.oz + sdz(k);
    return M.W[j] * (M.inv[row][0] + M.inv[row][1] * rx + M.inv[row][2] * ry + M.inv[row][3] * rz);
}

__device__ __forceinline__ int mls_node_g(const MemberDev& d, const MlsG& M, int k) {
    const int dx = sdx(k), dy = sdy(k), dz = sdz(k);
    return M.base >= 0 ? M.base + dx + d.NX * (dy + d.NY * dz) : support_index(d, M.bx + dx, M.by + dy, M.bz + dz);
}

__device__ __forceinline__ float group_sum(float v, unsigned mask) {
#pragma unroll
    for (int o = 1; o < GL; o <<= 1) v += __shfl_xor_sync(mask, v, o);
    return v;
}

// F_p + F_tau of vertex v from its two probe records (Eqs. hydroForP,
// hydroForNu): -(p+ - p-) n A + (tau+ - tau-) . n A, plus the volume penalty
// (Eq. volFor) stored with them.
__device__ __forceinline__ void hydro_force(const float* __restrict__ probe, const float* __restrict__ nrm,
                                            const float* __restrict__ area, int v, float& Hx, float& Hy,
                                            float& Hz) {
    // the two 32-byte records of the vertex (16-byte aligned) in four vector loads
    const float4* r = reinterpret_cast<const float4*>(probe + (size_t)2 * v * PROBE_STRIDE);
    const float4 a0 = r[0], a1 = r[1], b0 = r[2], b1 = r[3];
    const float nx = nrm[3 * v], ny = nrm[3 * v + 1], nz = nrm[3 * v + 2], A = area[v];
    const float dp = a0.x - b0.x;
    const float t0 = a0.y - b0.y, t1 = a0.z - b0.z, t2 = a0.w - b0.w, t3 = a1.x - b1.x, t4 = a1.y - b1.y,
                t5 = a1.z - b1.z;
    const float kv = a1.w;   // volume penalty k_v (1 - V/V0) A of soft capsules
    Hx = (-dp * nx + t0 * nx + t3 * ny + t4 * nz) * A + kv * nx;
    Hy = (-dp * ny + t3 * nx + t1 * ny + t5 * nz) * A + kv * ny;
    Hz = (-dp * nz + t4 * nx + t5 * ny + t2 * nz) * A + kv * nz;
}

// ---------------------------------------------------------------------------
// Stretching (Eq. strainFor) and bending of every hinge of soft capsules.
// Bending is -grad of k_b [1 - cos(theta - theta0)], the potential whose
// gradient carries the beta_b = k_b sin(theta - theta0)/sin(theta) factor of
// Eq. bendFor; theta is the signed angle between the outward normals.
// ---------------------------------------------------------------------------
// one vector reduction per vertex (the force array is padded to float4)
__device__ __forceinline__ void add_force(float* F, int v, f3 a) {
    atomicAdd(reinterpret_cast<float4*>(F) + v, make_float4(a.x, a.y, a.z, 0.f));
}

// ---------------------------------------------------------------------------
// Hinge forces (stretching of edge v2-v3, Eq. strainFor; bending of the hinge
// (v1, v2, v3, v4) as -grad of k_b [1 - cos(theta - theta0)], the potential
// whose gradient carries the beta_b = k_b sin(theta - theta0)/sin(theta)
// factor of Eq. bendFor, theta the signed angle between the outward normals),
// written once for a scalar type T: float for the forward step, and dual
// numbers (value, tangent) for the adjoint, where one evaluation with the
// tangent lambda_F at the four vertices gives d F / d x . lambda_F, which is
// the adjoint product because d F / d x = -Hessian is symmetric.
// ---------------------------------------------------------------------------
struct dual {
    float v, d;
};
__device__ __forceinline__ dual operator+(dual a, dual b) { return {a.v + b.v, a.d + b.d}; }
__device__ __forceinline__ dual operator-(dual a, dual b) { return {a.v - b.v, a.d - b.d}; }
__device__ __forceinline__ dual operator-(dual a) { return {-a.v, -a.d}; }
__device__ __forceinline__ dual operator-(dual a, float b) { return {a.v - b, a.d}; }
__device__ __forceinline__ dual operator+(dual a, float b) { return {a.v + b, a.d}; }
__device__ __forceinline__ dual operator*(dual a, dual b) { return {a.v * b.v, a.d * b.v + a.v * b.d}; }
__device__ __forceinline__ dual operator*(dual a, float b) { return {a.v * b, a.d * b}; }
__device__ __forceinline__ dual operator*(float a, dual b) { return {a * b.v, a * b.d}; }
__device__ __forceinline__ dual operator/(dual a, dual b) {
    const float q = a.v / b.v;
    return {q, (a.d - q * b.d) / b.v};
}
__device__ __forceinline__ dual operator/(float a, dual b) {
    const float q = a / b.v;
    return {q, -q * b.d / b.v};
}
__device__ __forceinline__ float tsqrt(float a) { return sqrtf(a); }
__device__ __forceinline__ dual tsqrt(dual a) {
    const float s = sqrtf(a.v);
    return {s, 0.5f * a.d / s};
}
__device__ __forceinline__ float tsin(float a) { return sinf(a); }
__device__ __forceinline__ dual tsin(dual a) { return {sinf(a.v), cosf(a.v) * a.d}; }
__device__ __forceinline__ float tatan2(float s, float c) { return atan2f(s, c); }
__device__ __forceinline__ dual tatan2(dual s, dual c) {
    return {atan2f(s.v, c.v), (c.v * s.d - s.v * c.d) / (s.v * s.v + c.v * c.v)};
}

template <typename T>
struct v3 {
    T x, y, z;
};
template <typename T>
__device__ __forceinline__ v3<T> sub(v3<T> a, v3<T> b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
template <typename T>
__device__ __forceinline__ v3<T> crs(v3<T> a, v3<T> b) {
    return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
template <typename T>
__device__ __forceinline__ T dot3(v3<T> a, v3<T> b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
template <typename T, typename S>
__device__ __forceinline__ v3<T> scl(v3<T> a, S s) { return {a.x * s, a.y * s, a.z * s}; }

// Forces on v1..v4 of a hinge from the positions relative to v2:
// a = x1 - x2, c = x3 - x2, dd = x4 - x2.
template <typename T>
__device__ __forceinline__ void hinge_forces(v3<T> a, v3<T> c, v3<T> dd, float ks, float l0, float kb, float th0,
                                             v3<T>& F1, v3<T>& F2, v3<T>& F3, v3<T>& F4) {
    // stretching on the edge (v2, v3): F_2 = -k (l - l0) r_23 / l, r_23 = v2 - v3
    const v3<T> r23 = scl(c, -1.f);
    const T l = tsqrt(dot3(r23, r23));
    const v3<T> Fs = scl(r23, -ks * (l - l0) / l);
    // bending on the hinge (v1, v2, v3, v4)
    const v3<T> nA = crs(scl(a, -1.f), sub(c, a));
    const v3<T> nB = crs(sub(c, dd), scl(dd, -1.f));
    const T L = l;
    const v3<T> eh = scl(c, 1.f / L);
    const T th = tatan2(dot3(crs(nA, nB), eh), dot3(nA, nB));
    const T k = kb * tsin(th - th0);
    const v3<T> gA = scl(nA, 1.f / dot3(nA, nA));
    const v3<T> gB = scl(nB, 1.f / dot3(nB, nB));
    const v3<T> u1 = scl(gA, L);
    const v3<T> u4 = scl(gB, L);
    const T pa = dot3(sub(a, c), eh), pd = dot3(sub(dd, c), eh);
    const v3<T> u2 = {pa * gA.x + pd * gB.x, pa * gA.y + pd * gB.y, pa * gA.z + pd * gB.z};
    const T qa = dot3(a, eh), qd = dot3(dd, eh);
    const v3<T> u3 = {-(qa * gA.x + qd * gB.x), -(qa * gA.y + qd * gB.y), -(qa * gA.z + qd * gB.z)};
    F1 = scl(u1, k);
    F2 = {k * u2.x + Fs.x, k * u2.y + Fs.y, k * u2.z + Fs.z};
    F3 = {k * u3.x - Fs.x, k * u3.y - Fs.y, k * u3.z - Fs.z};
    F4 = scl(u4, k);
}

}  // namespace ibl
