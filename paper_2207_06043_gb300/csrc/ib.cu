// Immersed-boundary and structure kernels: per-capsule geometry, the MLS
// interpolate/force/spread pass with the probe stresses and volume penalty (one
// thread per Lagrangian marker), per-hinge stretching + bending, inter-body
// repulsion on a cell list, and the Verlet / Newton-Euler update with the
// damage rule.
#include <climits>

#include "lbm_device.cuh"

namespace ibl {


constexpr float SUPPORT_SIDE = 2.6f;   // 2 r_w (Section "No-slip conditions for moving immersed boundaries")
constexpr float ALPHA = 0.3f;          // Eq. intKernel
constexpr double PIVOT_TOL = 1e-10;    // singular moment matrix -> nearest fluid node
constexpr unsigned FULL = 0xffffffffu;
constexpr uint32_t STOP = ST_DAMAGED | ST_NONFINITE;

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

// Support node k (0..26) of the point (X, Y, Z): the 3x3x3 block around the
// nearest node (round half up), in user coordinates; node is the padded index
// (-1 outside the domain), fluid false for solid or outside nodes.
__device__ __forceinline__ void support_node(const MemberDev& d, const uint8_t* __restrict__ tag, double X, double Y,
                                             double Z, int k, int& node, float& rx, float& ry, float& rz,
                                             bool& fluid) {
    const int bx = (int)floor(X + 0.5), by = (int)floor(Y + 0.5), bz = (int)floor(Z + 0.5);
    int cx = bx + (k % 3) - 1, cy = by + (k / 3) % 3 - 1, cz = bz + k / 9 - 1;
    rx = (float)((double)cx - X);
    ry = (float)((double)cy - Y);
    rz = (float)((double)cz - Z);
    bool ok = k < 27;
    if (d.per & 1) cx = ((cx % d.nx) + d.nx) % d.nx; else ok = ok && cx >= 0 && cx < d.nx;
    if (d.per & 2) cy = ((cy % d.ny) + d.ny) % d.ny; else ok = ok && cy >= 0 && cy < d.ny;
    if (d.per & 4) cz = ((cz % d.nz) + d.nz) % d.nz; else ok = ok && cz >= 0 && cz < d.nz;
    node = ok ? (cx + d.px) + d.NX * ((cy + d.py) + d.NY * (cz + d.pz)) : -1;
    fluid = ok && !(tag[d.node_off + node] & TAG_SOLID);
}

// Eq. intKernel with r normalised by the support side.
__device__ __forceinline__ float mls_weight(bool fluid, float rx, float ry, float rz) {
    const float r = sqrtf(rx * rx + ry * ry + rz * rz) * (1.f / SUPPORT_SIDE);
    const float s = r * (1.f / ALPHA);
    return (fluid && r <= 1.f) ? expf(-s * s) : 0.f;
}

// Column j of A^{-1} for the symmetric 4x4 moment matrix by L D L^T in FP64;
// good = every pivot above PIVOT_TOL * A00.
__device__ void ldlt_column(const double A[4][4], int j, double col[4], bool& good) {
    const double d0 = A[0][0];
    good = d0 > 0.0;
    const double s0 = d0 > 0.0 ? d0 : 1.0;
    const double L10 = A[1][0] / s0, L20 = A[2][0] / s0, L30 = A[3][0] / s0;
    const double d1 = A[1][1] - L10 * L10 * d0;
    const double s1 = d1 != 0.0 ? d1 : 1.0;
    const double L21 = (A[2][1] - L20 * L10 * d0) / s1;
    const double L31 = (A[3][1] - L30 * L10 * d0) / s1;
    const double d2 = A[2][2] - L20 * L20 * d0 - L21 * L21 * d1;
    const double s2 = d2 != 0.0 ? d2 : 1.0;
    const double L32 = (A[3][2] - L30 * L20 * d0 - L31 * L21 * d1) / s2;
    const double d3 = A[3][3] - L30 * L30 * d0 - L31 * L31 * d1 - L32 * L32 * d2;
    const double tol = PIVOT_TOL * s0;
    good = good && d1 > tol && d2 > tol && d3 > tol;
    if (!good) { col[0] = col[1] = col[2] = col[3] = 0.0; return; }
    // L y = e_j
    double y0 = j == 0 ? 1.0 : 0.0;
    double y1 = (j == 1 ? 1.0 : 0.0) - L10 * y0;
    double y2 = (j == 2 ? 1.0 : 0.0) - L20 * y0 - L21 * y1;
    double y3 = (j == 3 ? 1.0 : 0.0) - L30 * y0 - L31 * y1 - L32 * y2;
    // D z = y ; L^T c = z
    const double z0 = y0 / d0, z1 = y1 / d1, z2 = y2 / d2, z3 = y3 / d3;
    col[3] = z3;
    col[2] = z2 - L32 * col[3];
    col[1] = z1 - L21 * col[2] - L31 * col[3];
    col[0] = z0 - L10 * col[1] - L20 * col[2] - L30 * col[3];
}

// Warp-cooperative MLS shape functions (Eq. l2norm with the linear basis
// p = [1, x - X, y - Y, z - Z]): lane k < 27 holds W_k and its offsets and
// receives phi_k = W_k (A^{-1} p_k)_0 and, if want_grad, the gradient weights
// W_k (A^{-1} p_k)_{1..3}.  Moments are summed in FP32 (marker-relative
// offsets), the 4x4 system is solved in FP64.  A singular system hands the
// whole marker to the support node of largest weight.
__device__ void mls_weights(float W, float rx, float ry, float rz, int lane, bool want_grad, float& phi,
                            float& gx, float& gy, float& gz) {
    float mo[10] = {W, W * rx, W * ry, W * rz, W * rx * rx, W * rx * ry, W * rx * rz, W * ry * ry, W * ry * rz,
                    W * rz * rz};
#pragma unroll
    for (int i = 0; i < 10; ++i) mo[i] = warp_sum(mo[i]);
    double col[4] = {0.0, 0.0, 0.0, 0.0};
    bool good = false;
    if (lane < 4) {
        const double A[4][4] = {{mo[0], mo[1], mo[2], mo[3]},
                                {mo[1], mo[4], mo[5], mo[6]},
                                {mo[2], mo[5], mo[7], mo[8]},
                                {mo[3], mo[6], mo[8], mo[9]}};
        ldlt_column(A, lane, col, good);
    }
    good = __shfl_sync(FULL, (int)good, 0) != 0;
    gx = gy = gz = 0.f;
    if (good) {
        float r0[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) r0[c] = (float)__shfl_sync(FULL, col[c], 0);
        phi = W * (r0[0] + r0[1] * rx + r0[2] * ry + r0[3] * rz);
        if (want_grad) {
            float r1[4], r2[4], r3[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                r1[c] = (float)__shfl_sync(FULL, col[c], 1);
                r2[c] = (float)__shfl_sync(FULL, col[c], 2);
                r3[c] = (float)__shfl_sync(FULL, col[c], 3);
            }
            gx = W * (r1[0] + r1[1] * rx + r1[2] * ry + r1[3] * rz);
            gy = W * (r2[0] + r2[1] * rx + r2[2] * ry + r2[3] * rz);
            gz = W * (r3[0] + r3[1] * rx + r3[2] * ry + r3[3] * rz);
        }
    } else {
        float best = W;
        int bl = lane;
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            const float ob = __shfl_xor_sync(FULL, best, o);
            const int ol = __shfl_xor_sync(FULL, bl, o);
            if (ob > best || (ob == best && ol < bl)) { best = ob; bl = ol; }
        }
        phi = (best > 0.f && lane == bl) ? 1.f : 0.f;
    }
    if (lane >= 27) { phi = 0.f; gx = gy = gz = 0.f; }
}

template <typename T>
__device__ __forceinline__ void node_state(const MemberDev& d, const T* __restrict__ f,
                                           const float* __restrict__ face_vel, int node, int parity, int zh_on,
                                           float& rho, float& ux, float& uy, float& uz) {
    int X, Y, Z;
    node_coords(d, node, X, Y, Z);
    float g[Q];
    load_pre<T>(d, f + d.f_off, node, X, Y, Z, parity, g);
    if (zh_on) apply_face(d, X, Y, Z, face_vel, g);
    moments_of(g, rho, ux, uy, uz);
}

// ---------------------------------------------------------------------------
// per-capsule geometry at x(t): vertex areas A_v = 1/3 sum of adjacent triangle
// areas, vertex normals = normalised area-weighted triangle normals, and the
// FP64 enclosed volume (full = 1 adds area, centroid and second moments)
// ---------------------------------------------------------------------------
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

__global__ void __launch_bounds__(256) k_geometry(const CapsuleDev* __restrict__ caps, CapsuleSums* __restrict__ sums,
                                                  const uint32_t* __restrict__ status, const double* __restrict__ x,
                                                  const int* __restrict__ tri, float* __restrict__ nrm,
                                                  float* __restrict__ area, int full) {
    extern __shared__ float sh[];
    __shared__ double red[32];
    const CapsuleDev& C = caps[blockIdx.x];
    if (!full && (status[C.member] & STOP)) return;
    const int nv = C.v_count, vb = C.v_begin;
    __shared__ int box[6];
    if (threadIdx.x < 6) box[threadIdx.x] = threadIdx.x < 3 ? INT_MAX : INT_MIN;
    for (int v = threadIdx.x; v < 4 * nv; v += blockDim.x) sh[v] = 0.f;
    const double rx0 = x[3 * vb], ry0 = x[3 * vb + 1], rz0 = x[3 * vb + 2];
    __syncthreads();
    {
        int lo[3] = {INT_MAX, INT_MAX, INT_MAX}, hi[3] = {INT_MIN, INT_MIN, INT_MIN};
        for (int v = vb + threadIdx.x; v < vb + nv; v += blockDim.x) {
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const double c = x[3 * v + a];
                const int f = isfinite(c) ? (int)fmax(fmin(floor(c), 1e9), -1e9) : 0;
                lo[a] = min(lo[a], f);
                hi[a] = max(hi[a], f + 1);
            }
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            atomicMin(&box[a], lo[a]);
            atomicMax(&box[3 + a], hi[a]);
        }
    }
    double acc[11];
#pragma unroll
    for (int i = 0; i < 11; ++i) acc[i] = 0.0;
    for (int t = C.t_begin + threadIdx.x; t < C.t_begin + C.t_count; t += blockDim.x) {
        const int ia = tri[3 * t], ib = tri[3 * t + 1], ic = tri[3 * t + 2];
        const double ax = x[3 * ia] - rx0, ay = x[3 * ia + 1] - ry0, az = x[3 * ia + 2] - rz0;
        const double bx = x[3 * ib] - rx0, by = x[3 * ib + 1] - ry0, bz = x[3 * ib + 2] - rz0;
        const double cx = x[3 * ic] - rx0, cy = x[3 * ic + 1] - ry0, cz = x[3 * ic + 2] - rz0;
        const double ux = bx - ax, uy = by - ay, uz = bz - az;
        const double vx = cx - ax, vy = cy - ay, vz = cz - az;
        const double Nx = uy * vz - uz * vy, Ny = uz * vx - ux * vz, Nz = ux * vy - uy * vx;
        const double ar = 0.5 * sqrt(Nx * Nx + Ny * Ny + Nz * Nz);
        const int ids[3] = {ia - vb, ib - vb, ic - vb};
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            float* p = sh + 4 * ids[j];
            atomicAdd(p, (float)(0.5 * Nx));
            atomicAdd(p + 1, (float)(0.5 * Ny));
            atomicAdd(p + 2, (float)(0.5 * Nz));
            atomicAdd(p + 3, (float)(ar / 3.0));
        }
        const double vol = (ax * (by * cz - bz * cy) + ay * (bz * cx - bx * cz) + az * (bx * cy - by * cx)) / 6.0;
        acc[0] += vol;
        if (full) {
            acc[1] += ar;
            const double sx = ax + bx + cx, sy = ay + by + cy, sz = az + bz + cz;
            acc[2] += vol * sx * 0.25; acc[3] += vol * sy * 0.25; acc[4] += vol * sz * 0.25;
            const double c20 = vol / 20.0;
            acc[5] += c20 * (ax * ax + bx * bx + cx * cx + sx * sx);
            acc[6] += c20 * (ay * ay + by * by + cy * cy + sy * sy);
            acc[7] += c20 * (az * az + bz * bz + cz * cz + sz * sz);
            acc[8] += c20 * (ax * ay + bx * by + cx * cy + sx * sy);
            acc[9] += c20 * (ax * az + bx * bz + cx * cz + sx * sz);
            acc[10] += c20 * (ay * az + by * bz + cy * cz + sy * sz);
        }
    }
    const int nacc = full ? 11 : 1;
    for (int i = 0; i < nacc; ++i) {
        const double s = block_sum_d(acc[i], red);
        if (threadIdx.x == 0) {
            CapsuleSums& S = sums[blockIdx.x];
            switch (i) {
                case 0: S.V = s; break;
                case 1: S.S = s; break;
                case 2: case 3: case 4: S.cen[i - 2] = s; break;
                default: S.M2[i - 5] = s; break;
            }
        }
    }
    if (threadIdx.x == 0 && full) {
        sums[blockIdx.x].ref[0] = rx0; sums[blockIdx.x].ref[1] = ry0; sums[blockIdx.x].ref[2] = rz0;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        sums[blockIdx.x].box_lo[threadIdx.x] = box[threadIdx.x];
        sums[blockIdx.x].box_hi[threadIdx.x] = box[3 + threadIdx.x];
    }
    for (int v = threadIdx.x; v < nv; v += blockDim.x) {
        const float a = sh[4 * v], b = sh[4 * v + 1], c = sh[4 * v + 2];
        const float inv = rsqrtf(a * a + b * b + c * c);
        nrm[3 * (vb + v)] = a * inv;
        nrm[3 * (vb + v) + 1] = b * inv;
        nrm[3 * (vb + v) + 2] = c * inv;
        area[vb + v] = sh[4 * v + 3];
    }
}

// ---------------------------------------------------------------------------
// IB pre-pass and marker forces (one thread per marker), all on the fluid
// solution at t (the populations before this step's collision):
//   Eq. uLag on u* = sum g e / rho, F_l = (U_b - U_l)/dt, Eq. bodyforce
//   spreading with c_l = A_l into the dense f_ib field (float atomics) and the
//   node's IB flag; u_v,0 = U_l (the tentative velocity of Eq. verletPos);
//   probes at x +- 1.2 n: p = rho/3 and tau = rho nu (grad u + grad u^T) from
//   the MLS fit (Eqs. hydroForP, hydroForNu); the volume penalty
//   k_v (1 - V/V0) n A (Eq. volFor, restoring sign) of soft capsules.
// Writes force (overwrite; hinge and repulsion kernels add to it) and uv0.
// ---------------------------------------------------------------------------

// Moments (rho, u* = sum g e / rho) of the current populations at every fluid
// node of each capsule's vertex bounding box grown by SHELL_MARGIN, which
// holds every support node of the marker and probe stencils (probes sit
// 1.2 dx off the surface, supports reach 1.5 dx further).  The IB kernel then
// reads one float4 per support node instead of 19 scattered populations.
// Overlapping boxes write identical values.
constexpr int SHELL_MARGIN = 4;
constexpr int SHELL_BLOCKS = 32;   // blocks per capsule

template <typename T>
__global__ void __launch_bounds__(256) k_shell(const MemberDev* __restrict__ mem, const T* __restrict__ f,
                                               const uint8_t* __restrict__ tag, const float* __restrict__ face_vel,
                                               const uint32_t* __restrict__ status, const CapsuleDev* __restrict__ caps,
                                               const CapsuleSums* __restrict__ sums, float4* __restrict__ macro,
                                               int parity, int zh_on) {
    const int c = blockIdx.x / SHELL_BLOCKS;
    const CapsuleDev& C = caps[c];
    if (status[C.member] & STOP) return;
    const MemberDev& d = mem[C.member];
    const int dims[3] = {d.nx, d.ny, d.nz};
    int lo[3], ext[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        int l = sums[c].box_lo[a] - SHELL_MARGIN, h = sums[c].box_hi[a] + SHELL_MARGIN;
        if ((d.per >> a) & 1) {
            h = min(h, l + dims[a] - 1);
        } else {
            l = max(l, 0);
            h = min(h, dims[a] - 1);
        }
        lo[a] = l;
        ext[a] = h - l + 1;
    }
    if (ext[0] <= 0 || ext[1] <= 0 || ext[2] <= 0) return;
    const long long total = (long long)ext[0] * ext[1] * ext[2];
    for (long long i = (blockIdx.x % SHELL_BLOCKS) * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)SHELL_BLOCKS * blockDim.x) {
        int cx = lo[0] + (int)(i % ext[0]);
        int cy = lo[1] + (int)((i / ext[0]) % ext[1]);
        int cz = lo[2] + (int)(i / ((long long)ext[0] * ext[1]));
        if (d.per & 1) cx = ((cx % d.nx) + d.nx) % d.nx;
        if (d.per & 2) cy = ((cy % d.ny) + d.ny) % d.ny;
        if (d.per & 4) cz = ((cz % d.nz) + d.nz) % d.nz;
        const int node = (cx + d.px) + d.NX * ((cy + d.py) + d.NY * (cz + d.pz));
        if (tag[d.node_off + node] & TAG_SOLID) continue;
        float rho, ux, uy, uz;
        node_state<T>(d, f, face_vel, node, parity, zh_on, rho, ux, uy, uz);
        macro[d.node_off + node] = make_float4(rho, ux, uy, uz);
    }
}

// MLS operator of one point: weights W_k of the 27 support nodes (Eq.
// intKernel) and the rows of A^{-1} (Eq. l2norm, basis [1, x-X, y-Y, z-Z]);
// moments summed in FP32, the 4x4 system factorised in FP64.  fallback >= 0:
// singular system, the whole point goes to support node `fallback`.
struct Mls {
    int bx, by, bz;
    float ox, oy, oz;       // base node minus point
    float W[27];
    float inv[4][4];
    int fallback;           // -1: regular; 0..26: nearest fluid node; 27: none
};

__device__ __forceinline__ int support_index(const MemberDev& d, int cx, int cy, int cz) {
    if (d.per & 1) cx = ((cx % d.nx) + d.nx) % d.nx; else if (cx < 0 || cx >= d.nx) return -1;
    if (d.per & 2) cy = ((cy % d.ny) + d.ny) % d.ny; else if (cy < 0 || cy >= d.ny) return -1;
    if (d.per & 4) cz = ((cz % d.nz) + d.nz) % d.nz; else if (cz < 0 || cz >= d.nz) return -1;
    return (cx + d.px) + d.NX * ((cy + d.py) + d.NY * (cz + d.pz));
}

__device__ __forceinline__ void mls_build(const MemberDev& d, const uint8_t* __restrict__ tag, double X, double Y,
                                          double Z, Mls& M) {
    M.bx = (int)floor(X + 0.5); M.by = (int)floor(Y + 0.5); M.bz = (int)floor(Z + 0.5);
    M.ox = (float)((double)M.bx - X); M.oy = (float)((double)M.by - Y); M.oz = (float)((double)M.bz - Z);
    float m0 = 0, m1 = 0, m2 = 0, m3 = 0, m11 = 0, m12 = 0, m13 = 0, m22 = 0, m23 = 0, m33 = 0;
    float best = 0.f;
    int bestk = 27;
#pragma unroll
    for (int k = 0; k < 27; ++k) {
        const int dx = k % 3 - 1, dy = (k / 3) % 3 - 1, dz = k / 9 - 1;
        const int node = support_index(d, M.bx + dx, M.by + dy, M.bz + dz);
        const bool fluid = node >= 0 && !(tag[d.node_off + node] & TAG_SOLID);
        const float rx = M.ox + dx, ry = M.oy + dy, rz = M.oz + dz;
        const float w = mls_weight(fluid, rx, ry, rz);
        M.W[k] = w;
        if (w > best) { best = w; bestk = k; }
        m0 += w; m1 += w * rx; m2 += w * ry; m3 += w * rz;
        m11 += w * rx * rx; m12 += w * rx * ry; m13 += w * rx * rz;
        m22 += w * ry * ry; m23 += w * ry * rz; m33 += w * rz * rz;
    }
    const double A[4][4] = {{m0, m1, m2, m3}, {m1, m11, m12, m13}, {m2, m12, m22, m23}, {m3, m13, m23, m33}};
    // L D L^T in FP64
    const double d0 = A[0][0];
    const double s0 = d0 > 0.0 ? d0 : 1.0;
    const double L10 = A[1][0] / s0, L20 = A[2][0] / s0, L30 = A[3][0] / s0;
    const double d1 = A[1][1] - L10 * L10 * d0;
    const double s1 = d1 != 0.0 ? d1 : 1.0;
    const double L21 = (A[2][1] - L20 * L10 * d0) / s1;
    const double L31 = (A[3][1] - L30 * L10 * d0) / s1;
    const double d2 = A[2][2] - L20 * L20 * d0 - L21 * L21 * d1;
    const double s2 = d2 != 0.0 ? d2 : 1.0;
    const double L32 = (A[3][2] - L30 * L20 * d0 - L31 * L21 * d1) / s2;
    const double d3 = A[3][3] - L30 * L30 * d0 - L31 * L31 * d1 - L32 * L32 * d2;
    const double tol = PIVOT_TOL * s0;
    const bool good = d0 > 0.0 && d1 > tol && d2 > tol && d3 > tol;
    if (!good) {
        M.fallback = best > 0.f ? bestk : 27;
        return;
    }
    M.fallback = -1;
    const double r0 = 1.0 / d0, r1 = 1.0 / d1, r2 = 1.0 / d2, r3 = 1.0 / d3;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const double y0 = j == 0 ? 1.0 : 0.0;
        const double y1 = (j == 1 ? 1.0 : 0.0) - L10 * y0;
        const double y2 = (j == 2 ? 1.0 : 0.0) - L20 * y0 - L21 * y1;
        const double y3 = (j == 3 ? 1.0 : 0.0) - L30 * y0 - L31 * y1 - L32 * y2;
        const double c3 = y3 * r3;
        const double c2 = y2 * r2 - L32 * c3;
        const double c1 = y1 * r1 - L21 * c2 - L31 * c3;
        const double c0 = y0 * r0 - L10 * c1 - L20 * c2 - L30 * c3;
        M.inv[0][j] = (float)c0; M.inv[1][j] = (float)c1; M.inv[2][j] = (float)c2; M.inv[3][j] = (float)c3;
    }
}

template <typename T>
__global__ void __launch_bounds__(128) k_ib(const MemberDev* __restrict__ mem, const T* __restrict__ f, uint8_t* __restrict__ tag,
                                            float* __restrict__ fib, const float* __restrict__ face_vel,
                                            const uint32_t* __restrict__ status, const int* __restrict__ v_cap,
                                            const CapsuleDev* __restrict__ caps, const CapsuleSums* __restrict__ sums,
                                            const double* __restrict__ x, const double* __restrict__ vel,
                                            const float* __restrict__ nrm, const float* __restrict__ area,
                                            float* __restrict__ force, float* __restrict__ uv0, int n_verts,
                                            const float4* __restrict__ macro) {
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= n_verts) return;
    const int cap = v_cap[l];
    const CapsuleDev& C = caps[cap];
    const int m = C.member;
    if (status[m] & STOP) return;
    const MemberDev& d = mem[m];
    const double X = x[3 * l], Y = x[3 * l + 1], Z = x[3 * l + 2];
    const float A = area[l];
    Mls M;
    // --- interpolation at the marker (Eq. uLag) ---
    mls_build(d, tag, X, Y, Z, M);
    float Ux = 0.f, Uy = 0.f, Uz = 0.f;
    float phi[27];
#pragma unroll 1
    for (int k = 0; k < 27; ++k) {
        const float rx = M.ox + (k % 3 - 1), ry = M.oy + ((k / 3) % 3 - 1), rz = M.oz + (k / 9 - 1);
        float p = M.fallback < 0 ? M.W[k] * (M.inv[0][0] + M.inv[0][1] * rx + M.inv[0][2] * ry + M.inv[0][3] * rz)
                                 : (M.fallback == k ? 1.f : 0.f);
        phi[k] = p;
        if (p != 0.f) {
            const int node = support_index(d, M.bx + (k % 3 - 1), M.by + ((k / 3) % 3 - 1), M.bz + (k / 9 - 1));
            float rho, ux, uy, uz;
            const float4 q = macro[d.node_off + node];
            rho = q.x; ux = q.y; uy = q.z; uz = q.w;
            Ux += p * ux; Uy += p * uy; Uz += p * uz;
        }
    }
    // --- direct forcing and spreading (Eq. bodyforce) ---
    const float Fx = (float)vel[3 * l] - Ux, Fy = (float)vel[3 * l + 1] - Uy, Fz = (float)vel[3 * l + 2] - Uz;
#pragma unroll 1
    for (int k = 0; k < 27; ++k) {
        if (phi[k] != 0.f) {
            const int node = support_index(d, M.bx + (k % 3 - 1), M.by + ((k / 3) % 3 - 1), M.bz + (k / 9 - 1));
            const float c = A * phi[k];
            const size_t gi = (size_t)d.node_off + node;
            float* p = fib + 3 * gi;
            atomicAdd(p, c * Fx);
            atomicAdd(p + 1, c * Fy);
            atomicAdd(p + 2, c * Fz);
            tag[gi] = TAG_IB;   // fluid node: its tag byte was 0 or TAG_IB
        }
    }
    // --- probes at x +- 1.2 n (Eqs. hydroForP, hydroForNu) ---
    const float nx = nrm[3 * l], ny = nrm[3 * l + 1], nz = nrm[3 * l + 2];
    float dp = 0.f, dt0 = 0.f, dt1 = 0.f, dt2 = 0.f, dt3 = 0.f, dt4 = 0.f, dt5 = 0.f;
#pragma unroll 1
    for (int s = 0; s < 2; ++s) {
        const double sg = s == 0 ? 1.2 : -1.2;
        mls_build(d, tag, X + sg * nx, Y + sg * ny, Z + sg * nz, M);
        float rP = 0.f, G[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
#pragma unroll 1
        for (int k = 0; k < 27; ++k) {
            if (M.W[k] > 0.f) {
                const float rx = M.ox + (k % 3 - 1), ry = M.oy + ((k / 3) % 3 - 1), rz = M.oz + (k / 9 - 1);
                float p, g0 = 0.f, g1 = 0.f, g2 = 0.f;
                if (M.fallback < 0) {
                    const float w = M.W[k];
                    p = w * (M.inv[0][0] + M.inv[0][1] * rx + M.inv[0][2] * ry + M.inv[0][3] * rz);
                    g0 = w * (M.inv[1][0] + M.inv[1][1] * rx + M.inv[1][2] * ry + M.inv[1][3] * rz);
                    g1 = w * (M.inv[2][0] + M.inv[2][1] * rx + M.inv[2][2] * ry + M.inv[2][3] * rz);
                    g2 = w * (M.inv[3][0] + M.inv[3][1] * rx + M.inv[3][2] * ry + M.inv[3][3] * rz);
                } else {
                    p = M.fallback == k ? 1.f : 0.f;
                }
                const int node = support_index(d, M.bx + (k % 3 - 1), M.by + ((k / 3) % 3 - 1), M.bz + (k / 9 - 1));
                float r, vx, vy, vz;
                const float4 q = macro[d.node_off + node];
                r = q.x; vx = q.y; vy = q.z; vz = q.w;
                rP += p * r;
                G[0][0] += g0 * vx; G[0][1] += g1 * vx; G[0][2] += g2 * vx;
                G[1][0] += g0 * vy; G[1][1] += g1 * vy; G[1][2] += g2 * vy;
                G[2][0] += g0 * vz; G[2][1] += g1 * vz; G[2][2] += g2 * vz;
            }
        }
        const float mu = rP * d.nu;
        const float sgn = s == 0 ? 1.f : -1.f;
        dp += sgn * rP * (1.f / 3.f);
        dt0 += sgn * mu * 2.f * G[0][0];
        dt1 += sgn * mu * 2.f * G[1][1];
        dt2 += sgn * mu * 2.f * G[2][2];
        dt3 += sgn * mu * (G[0][1] + G[1][0]);
        dt4 += sgn * mu * (G[0][2] + G[2][0]);
        dt5 += sgn * mu * (G[1][2] + G[2][1]);
    }
    float Hx = -dp * A * nx + (dt0 * nx + dt3 * ny + dt4 * nz) * A;
    float Hy = -dp * A * ny + (dt3 * nx + dt1 * ny + dt5 * nz) * A;
    float Hz = -dp * A * nz + (dt4 * nx + dt5 * ny + dt2 * nz) * A;
    if (!C.rigid) {
        const float kvol = (float)(C.kv * (1.0 - sums[cap].V / C.V0));
        Hx += kvol * A * nx;
        Hy += kvol * A * ny;
        Hz += kvol * A * nz;
    }
    force[3 * l] = Hx; force[3 * l + 1] = Hy; force[3 * l + 2] = Hz;
    uv0[3 * l] = Ux; uv0[3 * l + 1] = Uy; uv0[3 * l + 2] = Uz;
}

// ---------------------------------------------------------------------------
// Stretching (Eq. strainFor) and bending of every hinge of soft capsules.
// Bending is -grad of k_b [1 - cos(theta - theta0)], the potential whose
// gradient carries the beta_b = k_b sin(theta - theta0)/sin(theta) factor of
// Eq. bendFor; theta is the signed angle between the outward normals.
// ---------------------------------------------------------------------------
struct f3 { float x, y, z; };
__device__ __forceinline__ f3 sub(f3 a, f3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ f3 crs(f3 a, f3 b) { return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x}; }
__device__ __forceinline__ float dot3(f3 a, f3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ f3 scl(f3 a, float s) { return {a.x * s, a.y * s, a.z * s}; }
__device__ __forceinline__ void add_force(float* F, int v, f3 a) {
    atomicAdd(F + 3 * v, a.x); atomicAdd(F + 3 * v + 1, a.y); atomicAdd(F + 3 * v + 2, a.z);
}

__global__ void __launch_bounds__(256) k_edges(const int* __restrict__ hinge, const int* __restrict__ e_cap,
                                               const CapsuleDev* __restrict__ caps, const uint32_t* __restrict__ status,
                                               const double* __restrict__ x, const float* __restrict__ l0,
                                               const float* __restrict__ ks, const float* __restrict__ th0,
                                               const float* __restrict__ kb, float* __restrict__ force, int n_edges) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n_edges) return;
    const CapsuleDev& C = caps[e_cap[e]];
    if (C.rigid || (status[C.member] & STOP)) return;
    const int v1 = hinge[4 * e], v2 = hinge[4 * e + 1], v3 = hinge[4 * e + 2], v4 = hinge[4 * e + 3];
    const double ox = x[3 * v2], oy = x[3 * v2 + 1], oz = x[3 * v2 + 2];
    const f3 a = {(float)(x[3 * v1] - ox), (float)(x[3 * v1 + 1] - oy), (float)(x[3 * v1 + 2] - oz)};
    const f3 c = {(float)(x[3 * v3] - ox), (float)(x[3 * v3 + 1] - oy), (float)(x[3 * v3 + 2] - oz)};
    const f3 dd = {(float)(x[3 * v4] - ox), (float)(x[3 * v4 + 1] - oy), (float)(x[3 * v4 + 2] - oz)};
    // stretching on the edge (v2, v3): F_2 = -k (l - l0) r_23 / l, r_23 = v2 - v3
    const f3 r23 = scl(c, -1.f);
    const float l = sqrtf(dot3(r23, r23));
    const f3 Fs = scl(r23, -ks[e] * (l - l0[e]) / l);
    // bending on the hinge (v1, v2, v3, v4)
    const f3 nA = crs(scl(a, -1.f), sub(c, a));
    const f3 nB = crs(sub(c, dd), scl(dd, -1.f));
    const float L = l;
    const f3 eh = scl(c, 1.f / L);
    const float th = atan2f(dot3(crs(nA, nB), eh), dot3(nA, nB));
    const float k = kb[e] * sinf(th - th0[e]);
    const f3 gA = scl(nA, 1.f / dot3(nA, nA));
    const f3 gB = scl(nB, 1.f / dot3(nB, nB));
    const f3 u1 = scl(gA, L);
    const f3 u4 = scl(gB, L);
    const float pa = dot3(sub(a, c), eh), pd = dot3(sub(dd, c), eh);
    const f3 u2 = {pa * gA.x + pd * gB.x, pa * gA.y + pd * gB.y, pa * gA.z + pd * gB.z};
    const float qa = dot3(a, eh), qd = dot3(dd, eh);
    const f3 u3 = {-(qa * gA.x + qd * gB.x), -(qa * gA.y + qd * gB.y), -(qa * gA.z + qd * gB.z)};
    add_force(force, v1, scl(u1, k));
    add_force(force, v2, {k * u2.x + Fs.x, k * u2.y + Fs.y, k * u2.z + Fs.z});
    add_force(force, v3, {k * u3.x - Fs.x, k * u3.y - Fs.y, k * u3.z - Fs.z});
    add_force(force, v4, scl(u4, k));
}

// ---------------------------------------------------------------------------
// Inter-body repulsion (Eq. collision) for markers of different capsules
// closer than 2 dx, found on a uniform grid of 2 dx cells.
// ---------------------------------------------------------------------------
__global__ void k_cells_fill(const MemberDev* __restrict__ mem, const int* __restrict__ v_cap, const CapsuleDev* __restrict__ caps,
                             const uint32_t* __restrict__ status, uint32_t* __restrict__ status_new,
                             const double* __restrict__ x, int* __restrict__ count, int* __restrict__ items,
                             int n_verts) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n_verts) return;
    const int m = caps[v_cap[v]].member;
    const MemberDev& d = mem[m];
    if (!d.has_cells || (status[m] & STOP)) return;
    const int cx = min(max((int)floor(x[3 * v] * 0.5), 0), d.cnx - 1);
    const int cy = min(max((int)floor(x[3 * v + 1] * 0.5), 0), d.cny - 1);
    const int cz = min(max((int)floor(x[3 * v + 2] * 0.5), 0), d.cnz - 1);
    const long long idx = d.cell_off + cx + (long long)d.cnx * (cy + (long long)d.cny * cz);
    const int slot = atomicAdd(count + idx, 1);
    if (slot < CELL_CAP) items[idx * CELL_CAP + slot] = v;
    else atomicOr(status_new + m, ST_OVERFLOW);
}

__global__ void k_repulsion(const MemberDev* __restrict__ mem, const int* __restrict__ v_cap, const CapsuleDev* __restrict__ caps,
                            const uint32_t* __restrict__ status, const double* __restrict__ x,
                            const float* __restrict__ nrm, const int* __restrict__ count, const int* __restrict__ items,
                            float* __restrict__ force, int n_verts) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_verts) return;
    const int ci = v_cap[i];
    const int m = caps[ci].member;
    const MemberDev& d = mem[m];
    if (!d.has_cells || (status[m] & STOP)) return;
    const double X = x[3 * i], Y = x[3 * i + 1], Z = x[3 * i + 2];
    const int cx = min(max((int)floor(X * 0.5), 0), d.cnx - 1);
    const int cy = min(max((int)floor(Y * 0.5), 0), d.cny - 1);
    const int cz = min(max((int)floor(Z * 0.5), 0), d.cnz - 1);
    float acc = 0.f;
    for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                const int qx = cx + dx, qy = cy + dy, qz = cz + dz;
                if (qx < 0 || qy < 0 || qz < 0 || qx >= d.cnx || qy >= d.cny || qz >= d.cnz) continue;
                const long long idx = d.cell_off + qx + (long long)d.cnx * (qy + (long long)d.cny * qz);
                const int cnt = min(count[idx], CELL_CAP);
                for (int s = 0; s < cnt; ++s) {
                    const int j = items[idx * CELL_CAP + s];
                    if (v_cap[j] == ci) continue;
                    // the cutoff decides a discontinuous force: take it in FP64
                    const double rx = X - x[3 * j], ry = Y - x[3 * j + 1], rz = Z - x[3 * j + 2];
                    const double d2 = rx * rx + ry * ry + rz * rz;
                    if (d2 < 4.0) {
                        const float dist = sqrtf((float)d2);
                        acc += 1.f / (dist * dist * sqrtf(dist));
                    }
                }
            }
    if (acc > 0.f) {
        const float c = d.umax * (1.f / (8.f * 1.41421356237f)) * acc;
        force[3 * i] -= c * nrm[3 * i];
        force[3 * i + 1] -= c * nrm[3 * i + 1];
        force[3 * i + 2] -= c * nrm[3 * i + 2];
    }
}

// ---------------------------------------------------------------------------
// Structure update (one block per capsule): Verlet predictor / velocity /
// corrector for soft capsules (Eqs. verletPos, verletVel, verletPosC), or the
// Newton-Euler system with Eq. angularVelRig for rigid bodies; then the
// damage rule (an edge at twice its rest length) and a finiteness check.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_update(CapsuleDev* __restrict__ caps, CapsuleSums* __restrict__ sums,
                                                const uint32_t* __restrict__ status,
                                                uint32_t* __restrict__ status_new, double* __restrict__ x,
                                                double* __restrict__ x_prev, double* __restrict__ vel,
                                                const float* __restrict__ force, const float* __restrict__ uv0,
                                                const int* __restrict__ hinge, const float* __restrict__ l0) {
    __shared__ double red[32];
    __shared__ double sh_rig[16];
    CapsuleDev& C = caps[blockIdx.x];
    const int m = C.member;
    if (status[m] & STOP) return;
    const int vb = C.v_begin, nv = C.v_count;
    bool bad = false;
    if (!C.rigid) {
        const double mv = C.mv;
        for (int v = vb + threadIdx.x; v < vb + nv; v += blockDim.x) {
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const double acc = 0.5 * (double)force[3 * v + a] / mv;
                const double xt = x[3 * v + a];
                const double xp = xt + (double)uv0[3 * v + a] + acc;
                const double un = 1.5 * xp - 2.0 * xt + 0.5 * x_prev[3 * v + a];
                const double xn = xt + un + acc;
                x_prev[3 * v + a] = xt;
                x[3 * v + a] = xn;
                vel[3 * v + a] = un;
                bad |= !isfinite(xn);
            }
        }
    } else {
        const double xc0 = C.xc[0], xc1 = C.xc[1], xc2 = C.xc[2];
        double s[6] = {0, 0, 0, 0, 0, 0};
        for (int v = vb + threadIdx.x; v < vb + nv; v += blockDim.x) {
            const double fx = force[3 * v], fy = force[3 * v + 1], fz = force[3 * v + 2];
            const double rx = x[3 * v] - xc0, ry = x[3 * v + 1] - xc1, rz = x[3 * v + 2] - xc2;
            s[0] += fx; s[1] += fy; s[2] += fz;
            s[3] += ry * fz - rz * fy; s[4] += rz * fx - rx * fz; s[5] += rx * fy - ry * fx;
        }
        for (int i = 0; i < 6; ++i) {
            const double t = block_sum_d(s[i], red);
            if (threadIdx.x == 0) sh_rig[i] = t;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double u[3], w[3];
            for (int a = 0; a < 3; ++a) {
                u[a] = (2.0 / 3.0) * (2.0 * C.u1[a] - 0.5 * C.u2[a] + sh_rig[a] / C.mass);
                w[a] = (2.0 / 3.0) * (2.0 * C.w1[a] - 0.5 * C.w2[a] + sh_rig[3 + a] / C.inertia);
            }
            // Rodrigues rotation by the angle vector w (dt = 1)
            const double th = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
            double R[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
            if (th > 0.0) {
                const double kx = w[0] / th, ky = w[1] / th, kz = w[2] / th;
                const double sn = sin(th), cs1 = 1.0 - cos(th);
                const double K[9] = {0, -kz, ky, kz, 0, -kx, -ky, kx, 0};
                double K2[9];
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j)
                        K2[3 * i + j] = K[3 * i] * K[j] + K[3 * i + 1] * K[3 + j] + K[3 * i + 2] * K[6 + j];
                for (int i = 0; i < 9; ++i) R[i] += sn * K[i] + cs1 * K2[i];
            }
            for (int i = 0; i < 9; ++i) sh_rig[i] = R[i];
            for (int a = 0; a < 3; ++a) {
                sh_rig[9 + a] = u[a];
                C.u2[a] = C.u1[a]; C.u1[a] = u[a];
                C.w2[a] = C.w1[a]; C.w1[a] = w[a];
            }
            sh_rig[12] = w[0]; sh_rig[13] = w[1]; sh_rig[14] = w[2];
        }
        __syncthreads();
        const double ncx = xc0 + sh_rig[9], ncy = xc1 + sh_rig[10], ncz = xc2 + sh_rig[11];
        const double* R = sh_rig;
        for (int v = vb + threadIdx.x; v < vb + nv; v += blockDim.x) {
            const double rx = x[3 * v] - xc0, ry = x[3 * v + 1] - xc1, rz = x[3 * v + 2] - xc2;
            const double qx = R[0] * rx + R[1] * ry + R[2] * rz;
            const double qy = R[3] * rx + R[4] * ry + R[5] * rz;
            const double qz = R[6] * rx + R[7] * ry + R[8] * rz;
            x_prev[3 * v] = x[3 * v]; x_prev[3 * v + 1] = x[3 * v + 1]; x_prev[3 * v + 2] = x[3 * v + 2];
            x[3 * v] = ncx + qx; x[3 * v + 1] = ncy + qy; x[3 * v + 2] = ncz + qz;
            const double wx = sh_rig[12], wy = sh_rig[13], wz = sh_rig[14];
            vel[3 * v] = sh_rig[9] + (wy * qz - wz * qy);
            vel[3 * v + 1] = sh_rig[10] + (wz * qx - wx * qz);
            vel[3 * v + 2] = sh_rig[11] + (wx * qy - wy * qx);
            bad |= !(isfinite(x[3 * v]) && isfinite(x[3 * v + 1]) && isfinite(x[3 * v + 2]));
        }
        __syncthreads();
        if (threadIdx.x == 0) { C.xc[0] = ncx; C.xc[1] = ncy; C.xc[2] = ncz; }
    }
    __syncthreads();
    if (!C.rigid) {
        // l >= 2 l0 decided on squared lengths in FP64 (no square root or
        // division on the slow FP64 path); the reported stretch in FP32
        double mx = 0.0;
        bool broken = false;
        for (int e = C.e_begin + threadIdx.x; e < C.e_begin + C.e_count; e += blockDim.x) {
            const int a = hinge[4 * e + 1], b = hinge[4 * e + 2];
            const double dx = x[3 * a] - x[3 * b], dy = x[3 * a + 1] - x[3 * b + 1], dz = x[3 * a + 2] - x[3 * b + 2];
            const double d2 = dx * dx + dy * dy + dz * dz;
            const double l0e = (double)l0[e];
            broken |= d2 >= 4.0 * l0e * l0e;
            mx = fmax(mx, (double)(sqrtf((float)d2) / l0[e]));
        }
        if (broken) mx = fmax(mx, 2.0);
#pragma unroll
        for (int o = 16; o; o >>= 1) mx = fmax(mx, __shfl_xor_sync(FULL, mx, o));
        __syncthreads();
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t = fmax(t, red[w]);
            sums[blockIdx.x].max_stretch = t;
            if (t >= 2.0) atomicOr(status_new + m, ST_DAMAGED);
        }
    }
    const int anybad = __syncthreads_or(bad ? 1 : 0);
    if (anybad && threadIdx.x == 0) atomicOr(status_new + m, ST_NONFINITE);
}

// ---------------------------------------------------------------------------
// launches
// ---------------------------------------------------------------------------
cudaError_t launch_geometry(const DevState& d, int full, cudaStream_t s) {
    if (d.n_caps == 0) return cudaSuccess;
    const size_t smem = 16 * (size_t)d.max_nv;
    static size_t configured = 0;
    if (smem > 48 * 1024 && smem > configured) {
        cudaError_t e = cudaFuncSetAttribute(k_geometry, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured = smem;
    }
    k_geometry<<<d.n_caps, 256, smem, s>>>(d.caps, d.sums, d.status, d.x, d.tri, d.nrm, d.area, full);
    return cudaGetLastError();
}

template <typename T>
static cudaError_t ib_t(const DevState& d, int parity, int zh_on, cudaStream_t s) {
    k_shell<T><<<d.n_caps * SHELL_BLOCKS, 256, 0, s>>>(d.mem, (const T*)d.f, d.tag, d.face_vel, d.status, d.caps,
                                                       d.sums, d.macro, parity, zh_on);
    k_ib<T><<<(unsigned)((d.n_verts + 127) / 128), 128, 0, s>>>(d.mem, (const T*)d.f, d.tag, d.fib, d.face_vel, d.status,
                                                              d.v_cap, d.caps, d.sums, d.x, d.vel, d.nrm, d.area,
                                                              d.force, d.uv0, d.n_verts, d.macro);
    return cudaGetLastError();
}

cudaError_t launch_ib(const DevState& d, int parity, int zh_on, cudaStream_t s) {
    if (d.n_verts == 0) return cudaSuccess;
    switch (d.storage) {
        case 1: return ib_t<__half>(d, parity, zh_on, s);
        case 2: return ib_t<__nv_bfloat16>(d, parity, zh_on, s);
        default: return ib_t<float>(d, parity, zh_on, s);
    }
}

cudaError_t launch_edges(const DevState& d, cudaStream_t s) {
    if (!d.any_soft || d.n_edges == 0) return cudaSuccess;
    k_edges<<<(d.n_edges + 255) / 256, 256, 0, s>>>(d.hinge, d.e_cap, d.caps, d.status, d.x, d.l0, d.ks, d.th0, d.kb,
                                                     d.force, d.n_edges);
    return cudaGetLastError();
}

cudaError_t launch_repulsion(const DevState& d, cudaStream_t s) {
    if (!d.any_cells) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(d.cell_count, 0, sizeof(int) * d.n_cells, s);
    if (e != cudaSuccess) return e;
    const int blocks = (d.n_verts + 255) / 256;
    k_cells_fill<<<blocks, 256, 0, s>>>(d.mem, d.v_cap, d.caps, d.status, d.status_new, d.x, d.cell_count, d.cell_items,
                                        d.n_verts);
    k_repulsion<<<blocks, 256, 0, s>>>(d.mem, d.v_cap, d.caps, d.status, d.x, d.nrm, d.cell_count, d.cell_items, d.force,
                                       d.n_verts);
    return cudaGetLastError();
}

cudaError_t launch_update(const DevState& d, cudaStream_t s) {
    if (d.n_caps == 0) return cudaSuccess;
    k_update<<<d.n_caps, 256, 0, s>>>(d.caps, d.sums, d.status, d.status_new, d.x, d.x_prev, d.vel, d.force, d.uv0,
                                      d.hinge, d.l0);
    return cudaGetLastError();
}

}  // namespace ibl
