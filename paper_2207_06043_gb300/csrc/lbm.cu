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

// Missing population of every wall link for the next step (Eq. bbouzidi, with
// the q >= 1/2 branch re-derived by quadratic interpolation and the two-point
// / halfway fall-backs when upstream nodes are not fluid).  Reads the
// post-collision values of the step just done (parity pp) and writes the slot
// the next step (parity 1 - pp) reads.
template <typename T>
__device__ __forceinline__ void bfl_link(const MemberDev* __restrict__ mem, T* __restrict__ f,
                                         const uint32_t* __restrict__ l_node, const float* __restrict__ l_q, int l,
                                         uint32_t meta, int pp, float* __restrict__ tape_dvdq) {
    const int m = (int)(meta >> 8);
    const MemberDev& d = mem[m];
    const int i = (int)(meta & 31u);
    const bool ok1 = meta & 32u, ok2 = meta & 64u;
    const int ib = opp(i);
    const int xb = (int)l_node[l];
    const float q = l_q[l];
    // x_b + e_i (solid, inside the box), x_b - e_i and x_b - 2 e_i (read only
    // when fluid): constant offsets in a lattice without periodic axes, else
    // wrapped coordinates
    int xsN, m1N, m2N;
    if (d.per == 0) {
        const int o = lin_off(d, i);
        xsN = xb + o; m1N = xb - o; m2N = xb - 2 * o;
    } else {
        int X, Y, Z;
        node_coords(d, xb, X, Y, Z);
        const bool px = d.per & 1, py = d.per & 2, pz = d.per & 4;
        const int exi = ex(i), eyi = ey(i), ezi = ez(i);
        xsN = nbc(X, exi, d.NX, px) + d.NX * (nbc(Y, eyi, d.NY, py) + d.NY * nbc(Z, ezi, d.NZ, pz));
        const int X1 = nbc(X, -exi, d.NX, px), Y1 = nbc(Y, -eyi, d.NY, py), Z1 = nbc(Z, -ezi, d.NZ, pz);
        m1N = X1 + d.NX * (Y1 + d.NY * Z1);
        m2N = nbc(X1, -exi, d.NX, px) + d.NX * (nbc(Y1, -eyi, d.NY, py) + d.NY * nbc(Z1, -ezi, d.NZ, pz));
    }
    const size_t S = (size_t)d.S;
    const float ls = d.ld_scale;
    T* fm = f + d.f_off;
    float fi_b, fib_b, fi_1 = 0.f, fi_2 = 0.f, fib_1 = 0.f;
    if (pp == 0) {
        fi_b = Store<T>::ld(fm + ib * S + xb, ls);
        fib_b = Store<T>::ld(fm + i * S + xb, ls);
        if (ok1) {
            fi_1 = Store<T>::ld(fm + ib * S + m1N, ls);
            fib_1 = Store<T>::ld(fm + i * S + m1N, ls);
            if (ok2) fi_2 = Store<T>::ld(fm + ib * S + m2N, ls);
        }
    } else {
        fi_b = Store<T>::ld(fm + i * S + xsN, ls);
        fib_b = Store<T>::ld(fm + ib * S + m1N, ls);
        if (ok1) {
            fi_1 = Store<T>::ld(fm + i * S + xb, ls);
            fib_1 = Store<T>::ld(fm + ib * S + m2N, ls);
            if (ok2) fi_2 = Store<T>::ld(fm + i * S + m1N, ls);
        }
    }
    float v;
    if (q < 0.5f) {
        if (ok1 && ok2) v = q * (2.f * q + 1.f) * fi_b + (1.f - 4.f * q * q) * fi_1 - q * (1.f - 2.f * q) * fi_2;
        else if (ok1) v = 2.f * q * fi_b + (1.f - 2.f * q) * fi_1;
        else v = fi_b;
    } else {
        if (ok1) v = fi_b / (q * (2.f * q + 1.f)) + (2.f * q - 1.f) / q * fib_b + (1.f - 2.f * q) / (1.f + 2.f * q) * fib_1;
        else v = fi_b / (2.f * q) + (2.f * q - 1.f) / (2.f * q) * fib_b;
    }
    if (tape_dvdq) {
        // d v / d q of the rule just applied (the derivative of each branch in q)
        float dv;
        if (q < 0.5f) {
            if (ok1 && ok2) dv = (4.f * q + 1.f) * fi_b - 8.f * q * fi_1 - (1.f - 4.f * q) * fi_2;
            else if (ok1) dv = 2.f * (fi_b - fi_1);
            else dv = 0.f;
        } else {
            const float a = q * (2.f * q + 1.f);
            if (ok1) dv = -(4.f * q + 1.f) / (a * a) * fi_b + fib_b / (q * q) - 4.f / ((1.f + 2.f * q) * (1.f + 2.f * q)) * fib_1;
            else dv = (fib_b - fi_b) / (2.f * q * q);
        }
        tape_dvdq[l] = dv;
    }
    if (pp == 0) Store<T>::st(fm + i * S + xsN, v, d.st_scale);   // next step odd: read from n - e_ib
    else Store<T>::st(fm + ib * S + xb, v, d.st_scale);           // next step even: own slot
}

// Zou-He faces (Eq. extbound) after the stream and the wall fill of a step
// (parity pp done): every fluid node of a velocity or pressure face gathers
// its populations as the next step will (parity 1 - pp), takes the face rule,
// and writes the populations entering from outside the box back into the
// slots the next step reads.  Wall-link values filled by the BFL pass are
// among the populations the rule reads, and it replaces only those entering
// through the box face.
template <typename T>
__device__ __forceinline__ void face_node(const MemberDev* __restrict__ mem, T* __restrict__ f, int i, uint32_t meta,
                                          const uint32_t* __restrict__ fc_node, const float* __restrict__ face_vel,
                                          int pp, float* __restrict__ tape_rho) {
    const int m = (int)(meta >> 8), fc = (int)(meta & 7u);
    const MemberDev& d = mem[m];
    const int n = (int)fc_node[i];
    int X, Y, Z;
    node_coords(d, n, X, Y, Z);
    T* fm = f + d.f_off;
    const int parity = 1 - pp;
    float g[Q];
    load_pre<T>(d, fm, n, X, Y, Z, parity, g);
    const int nx = fc == 0 ? -1 : (fc == 1 ? 1 : 0);
    const int ny = fc == 2 ? -1 : (fc == 3 ? 1 : 0);
    const int nz = fc == 4 ? -1 : (fc == 5 ? 1 : 0);
    if (tape_rho) {
        // rho of the face rule: (1 + Sg) / (1 + u.n) on a velocity face, the
        // imposed density on a pressure face
        float Sg = 0.f;
#pragma unroll
        for (int k = 0; k < Q; ++k) {
            const int en = ex(k) * nx + ey(k) * ny + ez(k) * nz;
            Sg += (en == 0 ? 1.f : (en > 0 ? 2.f : 0.f)) * g[k];
        }
        float rho = d.face_rho[fc];
        if (d.face_kind[fc] == FACE_VELOCITY) {
            const float* u = face_vel + 3 * (d.face_off[fc] + face_index(d, fc, X, Y, Z));
            rho = (1.f + Sg) / (1.f + (u[0] * nx + u[1] * ny + u[2] * nz));
        }
        tape_rho[i] = rho;
    }
    apply_face(d, X, Y, Z, face_vel, g);
#pragma unroll
    for (int k = 0; k < Q; ++k) {
        if (ex(k) * nx + ey(k) * ny + ez(k) * nz < 0)
            Store<T>::st(fm + pre_slot(d, n, X, Y, Z, parity, k), g[k], d.st_scale);
    }
}

// The wall fill and the faces of a step in one launch.  Threads [0, n_face)
// take one face node each: first the wall links that start on it (in the
// order they are listed), then the face rule, which reads those values; the
// other threads take one wall link each and skip the links of face nodes
// (flag LINK_AT_FACE).  No other thread reads or writes the slots a face
// node's rule reads: each of them is written by at most one link.
template <typename T>
__global__ void __launch_bounds__(256, 6) k_walls(const MemberDev* __restrict__ mem, T* __restrict__ f,
                                               const uint32_t* __restrict__ l_node, const uint32_t* __restrict__ l_meta,
                                               const float* __restrict__ l_q, const uint32_t* __restrict__ status,
                                               int n_links, const uint32_t* __restrict__ fc_node,
                                               const uint32_t* __restrict__ fc_meta, const int* __restrict__ fc_lbeg,
                                               const int* __restrict__ fc_links, const float* __restrict__ face_vel,
                                               int n_face_nodes, int pp, float* __restrict__ tape_dvdq,
                                               float* __restrict__ tape_rho) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n_face_nodes) {
        const uint32_t meta = fc_meta[t];
        if (status[meta >> 8] & (ST_DAMAGED | ST_NONFINITE)) return;
        for (int j = fc_lbeg[t]; j < fc_lbeg[t + 1]; ++j) {
            const int l = fc_links[j];
            bfl_link<T>(mem, f, l_node, l_q, l, l_meta[l], pp, tape_dvdq);
        }
        face_node<T>(mem, f, t, meta, fc_node, face_vel, pp, tape_rho);
        return;
    }
    const int l = t - n_face_nodes;
    if (l >= n_links) return;
    const uint32_t meta = l_meta[l];
    if ((meta & LINK_AT_FACE) || (status[meta >> 8] & (ST_DAMAGED | ST_NONFINITE))) return;
    bfl_link<T>(mem, f, l_node, l_q, l, meta, pp, tape_dvdq);
}

template <typename T>
static cudaError_t walls_t(const DevState& d, int pp, cudaStream_t s, float* tape_dvdq, float* tape_rho) {
    const int n = d.n_links + d.n_face_nodes;
    if (n == 0) return cudaSuccess;
    k_walls<T><<<(n + 255) / 256, 256, 0, s>>>(d.mem, (T*)d.f, d.l_node, d.l_meta, d.l_q, d.status, d.n_links,
                                               d.fc_node, d.fc_meta, d.fc_lbeg, d.fc_links, d.face_vel,
                                               d.n_face_nodes, pp, tape_dvdq, tape_rho);
    return cudaGetLastError();
}

cudaError_t launch_walls(const DevState& d, int pp, cudaStream_t s, float* tape_dvdq, float* tape_rho) {
    switch (d.storage) {
        case 1: return walls_t<__half>(d, pp, s, tape_dvdq, tape_rho);
        case 2: return walls_t<__nv_bfloat16>(d, pp, s, tape_dvdq, tape_rho);
        default: return walls_t<float>(d, pp, s, tape_dvdq, tape_rho);
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
