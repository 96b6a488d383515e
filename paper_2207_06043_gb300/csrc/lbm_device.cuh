// Device helpers shared by the lattice and immersed-boundary kernels:
// AA-pattern addressing, Zou-He faces, BGK collision with Guo forcing.
#pragma once

#include "ibl_internal.cuh"

namespace ibl {


__device__ __forceinline__ void node_coords(const MemberDev& d, int n, int& X, int& Y, int& Z) {
    X = n % d.NX;
    const int r = n / d.NX;
    Y = r % d.NY;
    Z = r / d.NY;
}

// coordinate c + e on an axis of n nodes; periodic axes wrap, padded axes
// never leave [0, n) for interior nodes (the ghost layer absorbs the step)
__device__ __forceinline__ int nbc(int c, int e, int n, bool per) {
    int v = c + e;
    if (per) v = (v < 0) ? v + n : (v >= n ? v - n : v);
    return v;
}

struct Nbr {
    int xs[3], ys[3], zs[3];   // coordinate of node + e for e = -1, 0, +1
};

__device__ __forceinline__ Nbr neighbours(const MemberDev& d, int X, int Y, int Z) {
    Nbr b;
    const bool px = d.per & 1, py = d.per & 2, pz = d.per & 4;
    b.xs[0] = nbc(X, -1, d.NX, px); b.xs[1] = X; b.xs[2] = nbc(X, 1, d.NX, px);
    b.ys[0] = nbc(Y, -1, d.NY, py); b.ys[1] = Y; b.ys[2] = nbc(Y, 1, d.NY, py);
    b.zs[0] = nbc(Z, -1, d.NZ, pz); b.zs[1] = Z; b.zs[2] = nbc(Z, 1, d.NZ, pz);
    return b;
}

// Pre-collision populations of node n at a step of the given parity (AA
// pattern).  Even steps keep f_k at its own node in slot k; odd steps find it
// in slot opp(k) of the upstream node n - e_k.
template <typename T>
__device__ __forceinline__ void load_pre(const MemberDev& d, const T* __restrict__ fm, int n, int X, int Y,
                                         int Z, int parity, float g[Q]) {
    const size_t S = (size_t)d.S;
    const float ls = d.ld_scale;
    if (parity == 0) {
#pragma unroll
        for (int k = 0; k < Q; ++k) g[k] = Store<T>::ld(fm + k * S + n, ls);
    } else {
        const Nbr b = neighbours(d, X, Y, Z);
#pragma unroll
        for (int k = 0; k < Q; ++k) {
            const int src = b.xs[1 - ex(k)] + d.NX * (b.ys[1 - ey(k)] + d.NY * b.zs[1 - ez(k)]);
            g[k] = Store<T>::ld(fm + opp(k) * S + src, ls);
        }
    }
}

// Element offset of the slot from which a step of the given parity gathers
// population k of node n (the address load_pre reads).
__device__ __forceinline__ long long pre_slot(const MemberDev& d, int n, int X, int Y, int Z, int parity, int k) {
    if (parity == 0) return (long long)k * d.S + n;
    const bool px = d.per & 1, py = d.per & 2, pz = d.per & 4;
    const int src = nbc(X, -ex(k), d.NX, px) + d.NX * (nbc(Y, -ey(k), d.NY, py) + d.NY * nbc(Z, -ez(k), d.NZ, pz));
    return (long long)opp(k) * d.S + src;
}

// Post-collision populations of node n: even steps swap them into slot opp(k)
// of their own node, odd steps push them to slot k of n + e_k.
template <typename T>
__device__ __forceinline__ void store_post(const MemberDev& d, T* __restrict__ fm, int n, int X, int Y, int Z,
                                           int parity, const float g[Q]) {
    const size_t S = (size_t)d.S;
    const float ss = d.st_scale;
    if (parity == 0) {
#pragma unroll
        for (int k = 0; k < Q; ++k) Store<T>::st(fm + opp(k) * S + n, g[k], ss);
    } else {
        const Nbr b = neighbours(d, X, Y, Z);
#pragma unroll
        for (int k = 0; k < Q; ++k) {
            const int dst = b.xs[1 + ex(k)] + d.NX * (b.ys[1 + ey(k)] + d.NY * b.zs[1 + ez(k)]);
            Store<T>::st(fm + k * S + dst, g[k], ss);
        }
    }
}

// The same two accesses for a node that is neither on a box face nor on the
// wrap plane of a periodic axis: every neighbour is n + e_k in the padded
// layout (the ghost layer absorbs the step on non-periodic axes), so no
// coordinates are needed.
__device__ __forceinline__ int lin_off(const MemberDev& d, int k) {
    return ex(k) + d.NX * (ey(k) + d.NY * ez(k));
}

template <typename T>
__device__ __forceinline__ void load_pre_lin(const MemberDev& d, const T* __restrict__ fm, int n, int parity,
                                             float g[Q]) {
    const size_t S = (size_t)d.S;
    const float ls = d.ld_scale;
    if (parity == 0) {
#pragma unroll
        for (int k = 0; k < Q; ++k) g[k] = Store<T>::ld(fm + k * S + n, ls);
    } else {
#pragma unroll
        for (int k = 0; k < Q; ++k) g[k] = Store<T>::ld(fm + opp(k) * S + (n - lin_off(d, k)), ls);
    }
}

template <typename T>
__device__ __forceinline__ void store_post_lin(const MemberDev& d, T* __restrict__ fm, int n, int parity,
                                               const float g[Q]) {
    const size_t S = (size_t)d.S;
    const float ss = d.st_scale;
    if (parity == 0) {
#pragma unroll
        for (int k = 0; k < Q; ++k) Store<T>::st(fm + opp(k) * S + n, g[k], ss);
    } else {
#pragma unroll
        for (int k = 0; k < Q; ++k) Store<T>::st(fm + k * S + (n + lin_off(d, k)), g[k], ss);
    }
}

// Box face of a node (-1: none).  Nodes on two faces are solid by
// construction of the geometry.
__device__ __forceinline__ int face_of(const MemberDev& d, int X, int Y, int Z) {
    if (!(d.per & 1)) { if (X == 1) return 0; if (X == d.NX - 2) return 1; }
    if (!(d.per & 2)) { if (Y == 1) return 2; if (Y == d.NY - 2) return 3; }
    if (!(d.per & 4)) { if (Z == 1) return 4; if (Z == d.NZ - 2) return 5; }
    return -1;
}

__device__ __forceinline__ int face_index(const MemberDev& d, int face, int X, int Y, int Z) {
    const int x = X - d.px, y = Y - d.py, z = Z - d.pz;
    return face < 2 ? y + d.ny * z : (face < 4 ? x + d.nx * z : x + d.nx * y);
}

// Zou-He (Eq. extbound) on the populations g = f - w of a face node, written
// for any face through its outward normal n: with Sg = sum_{e.n=0} g +
// 2 sum_{e.n>0} g, rho (1 + u.n) = 1 + Sg; every population entering from
// outside (e.n < 0) becomes g_opp - rho u.n / 3 (e = -n) or
// g_opp - rho u.n / 6 + rho u.t / 6 - N_t (e = -n + t) with
// N_t = 1/2 sum_{e.n=0} g (e.t) - rho u.t / 3.
__device__ __forceinline__ void zou_he(float g[Q], int face, int kind, float rho_w, float uwx, float uwy,
                                       float uwz) {
    const int nx = face == 0 ? -1 : (face == 1 ? 1 : 0);
    const int ny = face == 2 ? -1 : (face == 3 ? 1 : 0);
    const int nz = face == 4 ? -1 : (face == 5 ? 1 : 0);
    float Sg = 0.f, Tx = 0.f, Ty = 0.f, Tz = 0.f;
#pragma unroll
    for (int k = 0; k < Q; ++k) {
        const int en = ex(k) * nx + ey(k) * ny + ez(k) * nz;
        const float c0 = en == 0 ? 1.f : 0.f;
        const float c = en == 0 ? 1.f : (en > 0 ? 2.f : 0.f);
        Sg += c * g[k];
        Tx += c0 * (float)ex(k) * g[k];
        Ty += c0 * (float)ey(k) * g[k];
        Tz += c0 * (float)ez(k) * g[k];
    }
    float rho, un, ux, uy, uz;
    if (kind == FACE_VELOCITY) {
        un = uwx * nx + uwy * ny + uwz * nz;
        rho = (1.f + Sg) / (1.f + un);
        ux = uwx; uy = uwy; uz = uwz;
    } else {
        rho = rho_w;
        un = (1.f + Sg) / rho - 1.f;
        ux = un * nx; uy = un * ny; uz = un * nz;
    }
    float out[Q];
#pragma unroll
    for (int k = 0; k < Q; ++k) {
        const int en = ex(k) * nx + ey(k) * ny + ez(k) * nz;
        const int tx = ex(k) + nx, ty = ey(k) + ny, tz = ez(k) + nz;
        float v;
        if (tx == 0 && ty == 0 && tz == 0) {
            v = g[opp(k)] - rho * un * (1.f / 3.f);
        } else {
            const float ut = ux * tx + uy * ty + uz * tz;
            const float Nt = 0.5f * (Tx * tx + Ty * ty + Tz * tz) - rho * ut * (1.f / 3.f);
            v = g[opp(k)] - rho * un * (1.f / 6.f) + rho * ut * (1.f / 6.f) - Nt;
        }
        out[k] = en < 0 ? v : g[k];
    }
#pragma unroll
    for (int k = 0; k < Q; ++k) g[k] = out[k];
}

__device__ __forceinline__ void apply_face(const MemberDev& d, int X, int Y, int Z,
                                           const float* __restrict__ face_vel, float g[Q]) {
    const int fc = face_of(d, X, Y, Z);
    if (fc < 0) return;
    const int kind = d.face_kind[fc];
    if (kind == FACE_NONE) return;
    float ux = 0.f, uy = 0.f, uz = 0.f;
    if (kind == FACE_VELOCITY) {
        const float* u = face_vel + 3 * (d.face_off[fc] + face_index(d, fc, X, Y, Z));
        ux = u[0]; uy = u[1]; uz = u[2];
    }
    zou_he(g, fc, kind, d.face_rho[fc], ux, uy, uz);
}

// BGK collision (Eq. evoleq) with f^eq of Eq. eqfunc and the Guo term of
// Eq. forcing, on g = f - w: rho = 1 + sum g, rho u = sum g e + F/2,
// g^eq = w [drho + rho (3 e.u + 9/2 (e.u)^2 - 3/2 u^2)],
// F_i = (1 - 1/(2 tau)) w [3 (e - u).F + 9 (e.u)(e.F)].
__device__ __forceinline__ void collide(float g[Q], float omega, float guo, float Fx, float Fy, float Fz,
                                        bool hasF) {
    float drho = 0.f, jx = 0.f, jy = 0.f, jz = 0.f;
#pragma unroll
    for (int k = 0; k < Q; ++k) {
        drho += g[k];
        if (ex(k) > 0) jx += g[k]; else if (ex(k) < 0) jx -= g[k];
        if (ey(k) > 0) jy += g[k]; else if (ey(k) < 0) jy -= g[k];
        if (ez(k) > 0) jz += g[k]; else if (ez(k) < 0) jz -= g[k];
    }
    const float rho = 1.f + drho;
    const float inv = __frcp_rn(rho);   // correctly rounded, as 1.f / rho
    const float ux = (jx + 0.5f * Fx) * inv;
    const float uy = (jy + 0.5f * Fy) * inv;
    const float uz = (jz + 0.5f * Fz) * inv;
    const float usq = 1.5f * (ux * ux + uy * uy + uz * uz);
    const float uF = ux * Fx + uy * Fy + uz * Fz;
    // rest population, then each pair (k, opp(k)) at once: e.u and e.F change
    // sign between the two, so f_eq shares drho + rho (9/2 (e.u)^2 - 3/2 u^2)
    // and the Guo term shares 9 (e.u)(e.F) - 3 u.F
    {
        const float geq = wgt(0) * (drho - rho * usq);
        float o = g[0] + omega * (geq - g[0]);
        if (hasF) o += guo * wgt(0) * (-3.f * uF);
        g[0] = o;
    }
#pragma unroll
    for (int k = 1; k < Q; ++k) {
        if (opp(k) < k) continue;
        const int kb = opp(k);
        const float eu = ex(k) * ux + ey(k) * uy + ez(k) * uz;
        const float c = drho + rho * (4.5f * eu * eu - usq);
        const float t = 3.f * rho * eu;
        const float w = wgt(k);
        float ok = g[k] + omega * (w * (c + t) - g[k]);
        float ob = g[kb] + omega * (w * (c - t) - g[kb]);
        if (hasF) {
            const float eF = ex(k) * Fx + ey(k) * Fy + ez(k) * Fz;
            const float s = 9.f * eu * eF - 3.f * uF, gw = guo * w;
            ok += gw * (s + 3.f * eF);
            ob += gw * (s - 3.f * eF);
        }
        g[k] = ok;
        g[kb] = ob;
    }
}

__device__ __forceinline__ void moments_of(const float g[Q], float& rho, float& ux, float& uy, float& uz) {
    float drho = 0.f, jx = 0.f, jy = 0.f, jz = 0.f;
#pragma unroll
    for (int k = 0; k < Q; ++k) {
        drho += g[k];
        jx += ex(k) * g[k];
        jy += ey(k) * g[k];
        jz += ez(k) * g[k];
    }
    rho = 1.f + drho;
    const float inv = 1.f / rho;
    ux = jx * inv; uy = jy * inv; uz = jz * inv;
}

}  // namespace ibl
