// Lattice kernels: fused collide + stream (AA pattern, in place), the sparse
// Bouzidi-Firdaouss-Lallemand wall fill and Zou-He face passes,
// initialisation and read-out.
#include <algorithm>
#include <type_traits>

#include "lbm_device.cuh"

// launch bounds of the register-gather lattice kernel (threads per block,
// minimum resident blocks per SM); the register budget is 64K / (threads *
// blocks)
#ifndef LBM_THREADS
#define LBM_THREADS 128
#endif
#ifndef LBM_MIN_BLOCKS
#define LBM_MIN_BLOCKS 12
#endif
// the batched form reads its lattice's descriptor from global memory and
// needs more registers
#ifndef LBM_MIN_BLOCKS_BATCHED
#define LBM_MIN_BLOCKS_BATCHED 8
#endif

namespace ibl {


// Start of a step: flags raised during the previous step take effect, and
// every lattice still running counts one more step.
// The capsules' volume sums and bounding boxes restart from zero / empty.
__global__ void k_step_begin(uint32_t* __restrict__ status, uint32_t* __restrict__ status_new,
                             int* __restrict__ counters, int n_mem, CapsuleSums* __restrict__ sums, int n_caps) {
    const int m = threadIdx.x;
    if (m < n_mem) {
        const uint32_t st = status[m] | status_new[m];
        status[m] = st;
        if (!(st & (ST_DAMAGED | ST_NONFINITE))) counters[m] += 1;
    }
    for (int c = threadIdx.x; c < n_caps; c += blockDim.x) {
        sums[c].V = 0.0;
        for (int a = 0; a < 3; ++a) {
            // the previous box's centre (any point serves: it only anchors
            // the radial bounds of this step's vertices)
            const int lo = sums[c].box_lo[a], hi = sums[c].box_hi[a];
            sums[c].rc[a] = lo <= hi ? 0.5 * ((double)lo + (double)hi) : 0.0;
            sums[c].rcf[a] = (float)sums[c].rc[a];
            sums[c].box_lo[a] = 0x7fffffff;
            sums[c].box_hi[a] = -0x7fffffff - 1;
        }
        sums[c].r2_lo = 0x7f800000;   // +inf
        sums[c].r2_hi = 0;
    }
}

cudaError_t launch_step_begin(const DevState& d, cudaStream_t s) {
    k_step_begin<<<1, MAX_MEMBERS, 0, s>>>(d.status, d.status_new, d.counters, d.n_members, d.sums, d.n_caps);
    return cudaGetLastError();
}

// One time step of every fluid node of every member (Eq. evoleq): gather the
// pre-collision populations (AA parity; the face and wall rules of the
// previous step already sit in the gathered slots), add the body force and
// the spread IB force (which is then cleared), collide, store.
// Work list: the fluid nodes of each lattice in ascending order, one warp per
// group of 32 (each lattice's list padded to whole groups), so no lane idles
// on a solid node and consecutive lanes mostly read consecutive addresses.
// Interior nodes (BORDER false) address every neighbour by a constant offset
// and need no coordinates (the ghost layer of non-periodic axes absorbs the
// steps off the box); nodes on the wrap plane of a periodic axis take the
// coordinate-based path in a launch of their own.  Each population slot is
// read and written by one node per step (AA pattern), so the two launches are
// independent.
// SINGLE: the context holds one lattice, whose descriptor arrives by value in
// the kernel's parameter bank.
template <typename T, bool SINGLE, bool BORDER>
__global__ void __launch_bounds__(LBM_THREADS, BORDER ? 4 : (SINGLE ? LBM_MIN_BLOCKS : LBM_MIN_BLOCKS_BATCHED))
k_lbm(const __grid_constant__ MemberDev d0, const MemberDev* __restrict__ mem, T* __restrict__ f,
      uint8_t* __restrict__ tag, float* __restrict__ fib, const float* __restrict__ face_vel,
      const uint32_t* __restrict__ status, const uint32_t* __restrict__ nodes, const int* __restrict__ group_mem,
      int n_groups, int n_blocks, int parity, float4* __restrict__ tape, float4* __restrict__ tape_F) {
    const int warps = blockDim.x >> 5, lane = threadIdx.x & 31;
    for (int b = blockIdx.x; b < n_blocks; b += gridDim.x) {
        const int gi = b * warps + (threadIdx.x >> 5);
        if (gi >= n_groups) continue;
        // the node index and the member arrive together; the list holds
        // fluid nodes only, so the populations' loads wait on nothing else
        const uint32_t nn = nodes[(size_t)gi * 32 + lane];
        const int m = SINGLE ? 0 : group_mem[gi];
        const MemberDev& d = SINGLE ? d0 : mem[m];
        if (nn == NO_NODE || (status[m] & (ST_DAMAGED | ST_NONFINITE))) continue;
        const int n = (int)nn;
        const long long gn = d.node_off + n;
        const uint8_t tg = tag[gn];
        T* fm = f + d.f_off;
        // the spread IB force is fetched together with the populations
        const bool ibn = tg & TAG_IB;
        float4 fv = make_float4(0.f, 0.f, 0.f, 0.f);
        if (ibn) fv = reinterpret_cast<const float4*>(fib)[gn];
        float g[Q];
        int X = 0, Y = 0, Z = 0;
        if (BORDER) {
            node_coords(d, n, X, Y, Z);
            load_pre<T>(d, fm, n, X, Y, Z, parity, g);
        } else {
            load_pre_lin<T>(d, fm, n, parity, g);
        }
        float Fx = d.F[0], Fy = d.F[1], Fz = d.F[2];
        bool hasF = d.hasF != 0;
        if (ibn) {
            Fx += fv.x; Fy += fv.y; Fz += fv.z;
            reinterpret_cast<float4*>(fib)[gn] = make_float4(0.f, 0.f, 0.f, 0.f);
            tag[gn] = tg & (uint8_t)~TAG_IB;
            hasF = true;
        }
        if (tape_F) tape_F[gn] = make_float4(fv.x, fv.y, fv.z, ibn ? 1.f : 0.f);
        if (tape) {
            float rho, ux, uy, uz;
            moments_of(g, rho, ux, uy, uz);
            const float ir = __frcp_rn(rho);
            tape[gn] = make_float4(rho, ux + 0.5f * Fx * ir, uy + 0.5f * Fy * ir, uz + 0.5f * Fz * ir);
        }
        collide(g, d.omega, d.guo, Fx, Fy, Fz, hasF);
        if (BORDER) store_post<T>(d, fm, n, X, Y, Z, parity, g);
        else store_post_lin<T>(d, fm, n, parity, g);
    }
}

// Equilibrium initial state (parity 0 layout) from user-layout rho[N], u[3N].
template <typename T>
__global__ void k_init(const MemberDev* __restrict__ mem, T* __restrict__ f, const uint8_t* __restrict__ tag, int m, const float* __restrict__ rho,
                       const float* __restrict__ u) {
    const MemberDev& d = mem[m];
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= d.N) return;
    int X, Y, Z;
    node_coords(d, n, X, Y, Z);
    float g[Q];
    const bool solid = tag[d.node_off + n] & TAG_SOLID;
    const int x = X - d.px, y = Y - d.py, z = Z - d.pz;
    float r = 1.f, ux = 0.f, uy = 0.f, uz = 0.f;
    if (!solid) {
        const long long un = x + (long long)d.nx * (y + (long long)d.ny * z);
        if (rho) r = rho[un];
        if (u) { ux = u[3 * un]; uy = u[3 * un + 1]; uz = u[3 * un + 2]; }
    }
    const float usq = 1.5f * (ux * ux + uy * uy + uz * uz);
#pragma unroll
    for (int k = 0; k < Q; ++k) {
        const float eu = ex(k) * ux + ey(k) * uy + ez(k) * uz;
        g[k] = solid ? 0.f : wgt(k) * ((r - 1.f) + r * (3.f * eu + 4.5f * eu * eu - usq));
    }
    T* fm = f + d.f_off;
#pragma unroll
    for (int k = 0; k < Q; ++k) Store<T>::st(fm + (size_t)k * d.S + n, g[k], d.st_scale);
}

// Macroscopic fields / populations of one member in user layout.
template <typename T>
__global__ void k_read(const MemberDev* __restrict__ mem, const T* __restrict__ f, const uint8_t* __restrict__ tag, const float* __restrict__ face_vel,
                       int m, int parity, float* __restrict__ rho, float* __restrict__ u,
                       float* __restrict__ gout) {
    const MemberDev& d = mem[m];
    const long long Nu = (long long)d.nx * d.ny * d.nz;
    const long long un = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (un >= Nu) return;
    const int x = (int)(un % d.nx), y = (int)((un / d.nx) % d.ny), z = (int)(un / ((long long)d.nx * d.ny));
    const int X = x + d.px, Y = y + d.py, Z = z + d.pz;
    const int n = X + d.NX * (Y + d.NY * Z);
    float g[Q];
    const bool solid = tag[d.node_off + n] & TAG_SOLID;
    if (solid) {
#pragma unroll
        for (int k = 0; k < Q; ++k) g[k] = 0.f;
    } else {
        load_pre<T>(d, f + d.f_off, n, X, Y, Z, parity, g);
    }
    if (gout) {
#pragma unroll
        for (int k = 0; k < Q; ++k) gout[k * Nu + un] = g[k];
    }
    if (rho || u) {
        float r = 0.f, ux = 0.f, uy = 0.f, uz = 0.f;
        if (!solid) {
            float drho = 0.f, jx = 0.f, jy = 0.f, jz = 0.f;
#pragma unroll
            for (int k = 0; k < Q; ++k) {
                drho += g[k]; jx += ex(k) * g[k]; jy += ey(k) * g[k]; jz += ez(k) * g[k];
            }
            r = 1.f + drho;
            ux = (jx + 0.5f * d.F[0]) / r;
            uy = (jy + 0.5f * d.F[1]) / r;
            uz = (jz + 0.5f * d.F[2]) / r;
        }
        if (rho) rho[un] = r;
        if (u) { u[3 * un] = ux; u[3 * un + 1] = uy; u[3 * un + 2] = uz; }
    }
}

template <typename T>
static cudaError_t lbm_t(const DevState& d, int parity, cudaStream_t s, float4* tape, float4* tape_F) {
    const int grid = d.grid_lbm > 0 ? d.grid_lbm : d.lbm_blocks;
    const bool one = d.n_members == 1;
    if (grid > 0) {
        if (one)
            k_lbm<T, true, false><<<grid, d.threads, 0, s>>>(d.h_mem[0], d.mem, (T*)d.f, d.tag, d.fib, d.face_vel,
                                                             d.status, d.nodes, d.group_mem, d.n_groups,
                                                             d.lbm_blocks, parity, tape, tape_F);
        else
            k_lbm<T, false, false><<<grid, d.threads, 0, s>>>(d.h_mem[0], d.mem, (T*)d.f, d.tag, d.fib, d.face_vel,
                                                              d.status, d.nodes, d.group_mem, d.n_groups,
                                                              d.lbm_blocks, parity, tape, tape_F);
    }
    if (d.lbm_bblocks > 0) {
        if (one)
            k_lbm<T, true, true><<<d.lbm_bblocks, d.threads, 0, s>>>(d.h_mem[0], d.mem, (T*)d.f, d.tag, d.fib,
                                                                     d.face_vel, d.status, d.bnodes, d.bgroup_mem,
                                                                     d.n_bgroups, d.lbm_bblocks, parity, tape, tape_F);
        else
            k_lbm<T, false, true><<<d.lbm_bblocks, d.threads, 0, s>>>(d.h_mem[0], d.mem, (T*)d.f, d.tag, d.fib,
                                                                      d.face_vel, d.status, d.bnodes, d.bgroup_mem,
                                                                      d.n_bgroups, d.lbm_bblocks, parity, tape, tape_F);
    }
    return cudaGetLastError();
}

int lbm_max_threads() { return LBM_THREADS; }

cudaError_t launch_lbm(const DevState& d, int parity, cudaStream_t s, float4* tape_rhou, float4* tape_F) {
    switch (d.storage) {
        case 1: return lbm_t<__half>(d, parity, s, tape_rhou, tape_F);
        case 2: return lbm_t<__nv_bfloat16>(d, parity, s, tape_rhou, tape_F);
        default: return lbm_t<float>(d, parity, s, tape_rhou, tape_F);
    }
}


template <typename T>
static cudaError_t init_t(const DevState& d, int m, const float* rho, const float* u, cudaStream_t s) {
    const int N = d.h_mem[m].N;
    k_init<T><<<(N + 255) / 256, 256, 0, s>>>(d.mem, (T*)d.f, d.tag, m, rho, u);
    return cudaGetLastError();
}

cudaError_t launch_init_member(const DevState& d, int m, const float* rho, const float* u, cudaStream_t s) {
    switch (d.storage) {
        case 1: return init_t<__half>(d, m, rho, u, s);
        case 2: return init_t<__nv_bfloat16>(d, m, rho, u, s);
        default: return init_t<float>(d, m, rho, u, s);
    }
}

template <typename T>
static cudaError_t read_t(const DevState& d, int m, int parity, float* rho, float* u, float* g,
                          cudaStream_t s) {
    const MemberDev& md = d.h_mem[m];
    const long long Nu = (long long)md.nx * md.ny * md.nz;
    k_read<T><<<(unsigned)((Nu + 255) / 256), 256, 0, s>>>(d.mem, (const T*)d.f, d.tag, d.face_vel, m, parity, rho,
                                                           u, g);
    return cudaGetLastError();
}

cudaError_t launch_read(const DevState& d, int m, int parity, float* rho, float* u, float* g,
                        cudaStream_t s) {
    switch (d.storage) {
        case 1: return read_t<__half>(d, m, parity, rho, u, g, s);
        case 2: return read_t<__nv_bfloat16>(d, m, parity, rho, u, g, s);
        default: return read_t<float>(d, m, parity, rho, u, g, s);
    }
}

}  // namespace ibl
