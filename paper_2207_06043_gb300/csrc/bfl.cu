// The wall fill and the Zou-He faces of a time step, in one launch: the
// missing population of every wall link by the quadratic bounce-back
// (Section "Boundary conditions on fixed bodies", Eq. bbouzidi) and the
// entering populations of every fluid node on a velocity or pressure face
// (Eq. extbound), after the lattice kernel and before the next step.
#include <cstdint>

#include "lbm_device.cuh"

namespace ibl {

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
    // each branch of the rule reads three of the five values: q < 1/2 the
    // outgoing population at x_b, x_b - e_i and x_b - 2 e_i; q >= 1/2 the
    // outgoing one at x_b and the incoming ones at x_b and x_b - e_i
    const bool near = q < 0.5f;
    float fi_b, fib_b = 0.f, fi_1 = 0.f, fi_2 = 0.f, fib_1 = 0.f;
    if (pp == 0) {
        fi_b = Store<T>::ld(fm + ib * S + xb, ls);
        if (near) {
            if (ok1) {
                fi_1 = Store<T>::ld(fm + ib * S + m1N, ls);
                if (ok2) fi_2 = Store<T>::ld(fm + ib * S + m2N, ls);
            }
        } else {
            fib_b = Store<T>::ld(fm + i * S + xb, ls);
            if (ok1) fib_1 = Store<T>::ld(fm + i * S + m1N, ls);
        }
    } else {
        fi_b = Store<T>::ld(fm + i * S + xsN, ls);
        if (near) {
            if (ok1) {
                fi_1 = Store<T>::ld(fm + i * S + xb, ls);
                if (ok2) fi_2 = Store<T>::ld(fm + i * S + m1N, ls);
            }
        } else {
            fib_b = Store<T>::ld(fm + ib * S + m1N, ls);
            if (ok1) fib_1 = Store<T>::ld(fm + ib * S + m2N, ls);
        }
    }
    float v;
    if (near) {
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
        if (near) {
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
    const int nx = fc == 0 ? -1 : (fc == 1 ? 1 : 0);
    const int ny = fc == 2 ? -1 : (fc == 3 ? 1 : 0);
    const int nz = fc == 4 ? -1 : (fc == 5 ? 1 : 0);
    // the populations the rule reads: those not entering from outside
    // (e.n >= 0); the entering ones it replaces without reading
    float g[Q];
#pragma unroll
    for (int k = 0; k < Q; ++k)
        g[k] = ex(k) * nx + ey(k) * ny + ez(k) * nz < 0
                   ? 0.f
                   : Store<T>::ld(fm + pre_slot(d, n, X, Y, Z, parity, k), d.ld_scale);
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

}  // namespace ibl
