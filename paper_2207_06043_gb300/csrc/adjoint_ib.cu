// Discrete adjoint of the capsule part of the coupled step (reverse of the
// IB pre-pass, the membrane, volume and probe forces and the Verlet update of
// soft capsules), run after the lattice adjoint of the same step t:
//
//   forward step t (Reading T1 order):
//     geometry   A_l, n_l, V from x(t)
//     markers    U_l = sum_k phi_k(x_l) u*_k,  F_l = v_l - U_l,
//                f_ib_k += A_l phi_k(x_l) F_l                       (Eqs. uLag, bodyforce)
//     forces     F_tot = F_sb(x; 1/Ca) + kv (1 - V/V0) A n + F_h    (Eqs. strainFor .. hydroForNu)
//     Verlet     x' = x/2 + x_prev/2 + 3/2 U + 5/2 a,  v' = -x/2 + x_prev/2 + 3/2 U + 3/2 a,
//                x_prev' = x,  a = F_tot / (2 m_v)                  (Eqs. verletPos .. verletPosC)
//     lattice    f(t+1) from f(t) and f_ib
//
//   reverse step t, given the adjoints (lx, lxp, lv) of (x, x_prev, v) at t+1,
//   lambda_F of every IB node (lattice adjoint) and the population adjoint
//   lam_out of f(t) (lattice part):
//     k_adj_verlet    lU = 3/2 (lx + lv), lF = (5/2 lx + 3/2 lv)/(2 m_v),
//                     lx <- lx/2 - lv/2 + lxp, lxp <- (lx + lv)/2
//     k_adj_hinges    lx += dF_sb/dx . lF (dual numbers), d J/d Ca gains -F_sb.lF / Ca
//     k_adj_probes    the probe stresses: (lambda_rho, lambda_u*) of the support
//                     nodes, lx and ln through the probe point, ln and lA
//     k_adj_markers   the interpolation and spreading: lv, lx, lA, the
//                     support nodes' lambda_u*, and the volume penalty
//     k_adj_geometry  ln, lA and lambda_V back to lx through the triangles
//     k_adj_fold      lam_out += d(rho, u*)/df . (lambda_rho, lambda_u*) at the
//                     support nodes
// The moments (rho, u*) of f(t) come from the lattice tape, u* = u - F/(2 rho).
//
// MLS shape functions (Eq. l2norm, basis p = [1, x_k - P]): phi^j_k = W_k
// (A^-1 p_k)_j with A = sum_k W_k p_k p_k^T and W_k = exp(-|x_k - P|^2 /
// sigma^2), sigma = 2.6 * 0.3.  For row weights lambda_jk the product
// sum_jk lambda_jk d phi^j_k / d P is, with b^j = A^-1 sum_k lambda_jk W_k p_k,
// alpha_jk = (A^-1 p_k)_j and beta_jk = p_k . b^j,
//   sum_j sum_k (2 / sigma^2) (x_k - P) W_k alpha_jk (lambda_jk - beta_jk) + b^0_{1..3}
// (the terms through d p_k / d P cancel because A b^j reproduces the first
// moment of lambda_j, and sum_k W_k alpha_jk = delta_j0).  A singular stencil
// (nearest fluid node) does not depend on P.
#include "ib_device.cuh"

namespace ibl {

constexpr float INV_SIGMA2 = 1.f / (SUPPORT_SIDE * ALPHA * SUPPORT_SIDE * ALPHA);

struct AdjCap {
    float4* lx;        // adjoint of x (per vertex)
    float4* lxp;       // adjoint of x(t - dt)
    float4* lv;        // adjoint of the vertex velocity (the markers' U_b)
    float4* lU;        // adjoint of u_v,0 = U_l from the Verlet update
    float4* lF;        // adjoint of the total force
    float4* ln;        // adjoint of the vertex normal
    float* lA;         // adjoint of the vertex area
    float* snorm;      // |S_l|, the length of the unnormalised vertex normal
    double* lV;        // adjoint of the capsule volume (per capsule)
    float4* lfib;      // per node: lambda_F at the IB nodes (lattice adjoint)
    float4* lmac;      // per node: (lambda_rho, lambda_u*) of the support nodes
    double* acc_ca;    // sum over steps of F_sb . lF
};

__device__ __forceinline__ void add4(float4* p, float x, float y, float z, float w = 0.f) {
    atomicAdd(p, make_float4(x, y, z, w));
}

// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_adj_verlet(const CapsuleDev* __restrict__ caps, const int* __restrict__ v_cap,
                                                    AdjCap a, int n_verts) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n_verts) return;
    const float4 x = a.lx[v], xp = a.lxp[v], vv = a.lv[v];
    const float him = 0.5f / (float)caps[v_cap[v]].mv;
    a.lU[v] = make_float4(1.5f * (x.x + vv.x), 1.5f * (x.y + vv.y), 1.5f * (x.z + vv.z), 0.f);
    a.lF[v] = make_float4((2.5f * x.x + 1.5f * vv.x) * him, (2.5f * x.y + 1.5f * vv.y) * him,
                          (2.5f * x.z + 1.5f * vv.z) * him, 0.f);
    a.lx[v] = make_float4(0.5f * (x.x - vv.x) + xp.x, 0.5f * (x.y - vv.y) + xp.y, 0.5f * (x.z - vv.z) + xp.z, 0.f);
    a.lxp[v] = make_float4(0.5f * (x.x + vv.x), 0.5f * (x.y + vv.y), 0.5f * (x.z + vv.z), 0.f);
    a.lv[v] = make_float4(0.f, 0.f, 0.f, 0.f);
    a.ln[v] = make_float4(0.f, 0.f, 0.f, 0.f);
    a.lA[v] = 0.f;
}

// Per capsule: the volume and box sums restart, and the volume adjoint too.
__global__ void k_adj_geo_reset(CapsuleSums* __restrict__ sums, double* __restrict__ lV, int n_caps) {
    for (int c = threadIdx.x; c < n_caps; c += blockDim.x) {
        sums[c].V = 0.0;
        for (int k = 0; k < 3; ++k) {
            sums[c].box_lo[k] = 0x7fffffff;
            sums[c].box_hi[k] = -0x7fffffff - 1;
        }
        sums[c].r2_lo = 0x7f800000;
        sums[c].r2_hi = 0;
        lV[c] = 0.0;
    }
}

// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_adj_hinges(const int* __restrict__ hinge, const int* __restrict__ e_cap,
                                                    const CapsuleDev* __restrict__ caps, const float4* __restrict__ xm,
                                                    const float* __restrict__ l0, const float* __restrict__ ks,
                                                    const float* __restrict__ th0, const float* __restrict__ kb,
                                                    AdjCap a, int n_edges) {
    __shared__ double red[32];
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    double s = 0.0;
    if (e < n_edges && !caps[e_cap[e]].rigid) {
        const int4 hg = reinterpret_cast<const int4*>(hinge)[e];
        const f3 pa = mirror_diff(xm, hg.x, hg.y), pc = mirror_diff(xm, hg.z, hg.y), pd = mirror_diff(xm, hg.w, hg.y);
        const float4 t1 = a.lF[hg.x], t2 = a.lF[hg.y], t3 = a.lF[hg.z], t4 = a.lF[hg.w];
        const v3<dual> A = {{pa.x, t1.x - t2.x}, {pa.y, t1.y - t2.y}, {pa.z, t1.z - t2.z}};
        const v3<dual> C = {{pc.x, t3.x - t2.x}, {pc.y, t3.y - t2.y}, {pc.z, t3.z - t2.z}};
        const v3<dual> Dd = {{pd.x, t4.x - t2.x}, {pd.y, t4.y - t2.y}, {pd.z, t4.z - t2.z}};
        v3<dual> F1, F2, F3, F4;
        hinge_forces<dual>(A, C, Dd, ks[e], l0[e], kb[e], th0[e], F1, F2, F3, F4);
        add4(a.lx + hg.x, F1.x.d, F1.y.d, F1.z.d);
        add4(a.lx + hg.y, F2.x.d, F2.y.d, F2.z.d);
        add4(a.lx + hg.z, F3.x.d, F3.y.d, F3.z.d);
        add4(a.lx + hg.w, F4.x.d, F4.y.d, F4.z.d);
        s = (double)(F1.x.v * t1.x + F1.y.v * t1.y + F1.z.v * t1.z) +
            (double)(F2.x.v * t2.x + F2.y.v * t2.y + F2.z.v * t2.z) +
            (double)(F3.x.v * t3.x + F3.y.v * t3.y + F3.z.v * t3.z) +
            (double)(F4.x.v * t4.x + F4.y.v * t4.y + F4.z.v * t4.z);
    }
    const double t = block_sum_d(s, red);
    if (threadIdx.x == 0 && t != 0.0) atomicAdd(a.acc_ca, t);
}

// ---------------------------------------------------------------------------
// Moments of f(t) at a support node from the lattice tape: rho and
// u* = u - (F_body + f_ib) / (2 rho).
__device__ __forceinline__ float4 tape_macro(const MemberDev& d, const float4* __restrict__ tape,
                                             const float4* __restrict__ tape_F, int node) {
    const float4 t = tape[d.node_off + node];
    const float4 fi = tape_F[d.node_off + node];
    const float h = 0.5f / t.x;
    return make_float4(t.x, t.y - (d.F[0] + fi.x) * h, t.z - (d.F[1] + fi.y) * h, t.w - (d.F[2] + fi.z) * h);
}

// The moments a stencil reads at a support node: a fluid node's from the
// tape, a solid node's from the wall it lies in (rho = 1, u = 0; constants).
__device__ __forceinline__ float4 node_macro(const MemberDev& d, const uint8_t* __restrict__ tag,
                                             const float4* __restrict__ tape, const float4* __restrict__ tape_F,
                                             int node) {
    if (tag[d.node_off + node] & TAG_SOLID) return make_float4(1.f, 0.f, 0.f, 0.f);
    return tape_macro(d, tape, tape_F, node);
}

// The MLS product of the header comment for the lanes of one group: lam[j][s]
// are the row weights of this lane's support slots s (rows < NR), returns
// d/dP of sum_jk lam_jk phi^j_k (the same in every lane of the group).
template <int NR>
__device__ __forceinline__ f3 mls_vjp_g(const MlsG& M, const float (&lam)[NR][GS], int r, unsigned mask) {
    // b^j = A^-1 sum_k lam_jk W_k p_k
    float v[NR][4];
#pragma unroll
    for (int j = 0; j < NR; ++j) {
        v[j][0] = v[j][1] = v[j][2] = v[j][3] = 0.f;
#pragma unroll
        for (int s = 0; s < GS; ++s) {
            const int k = r + GL * s;
            if (k >= 27) continue;
            const float w = lam[j][s] * M.W[s];
            v[j][0] += w;
            v[j][1] += w * (M.ox + sdx(k));
            v[j][2] += w * (M.oy + sdy(k));
            v[j][3] += w * (M.oz + sdz(k));
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) v[j][c] = group_sum(v[j][c], mask);
    }
    float b[NR][4];
#pragma unroll
    for (int j = 0; j < NR; ++j)
#pragma unroll
        for (int c = 0; c < 4; ++c)
            b[j][c] = M.inv[c][0] * v[j][0] + M.inv[c][1] * v[j][1] + M.inv[c][2] * v[j][2] + M.inv[c][3] * v[j][3];
    float gx = 0.f, gy = 0.f, gz = 0.f;
#pragma unroll
    for (int s = 0; s < GS; ++s) {
        const int k = r + GL * s;
        if (k >= 27) continue;
        const float rx = M.ox + sdx(k), ry = M.oy + sdy(k), rz = M.oz + sdz(k);
        float term = 0.f;
#pragma unroll
        for (int j = 0; j < NR; ++j) {
            const float al = M.inv[j][0] + M.inv[j][1] * rx + M.inv[j][2] * ry + M.inv[j][3] * rz;
            const float be = b[j][0] + b[j][1] * rx + b[j][2] * ry + b[j][3] * rz;
            term += al * (lam[j][s] - be);
        }
        term *= 2.f * INV_SIGMA2 * M.W[s];
        gx += rx * term; gy += ry * term; gz += rz * term;
    }
    gx = group_sum(gx, mask) + b[0][1];
    gy = group_sum(gy, mask) + b[0][2];
    gz = group_sum(gz, mask) + b[0][3];
    return {gx, gy, gz};
}

// Probe at x + sg n (sg = +-1.2): p = rho_P / 3, tau = rho_P nu (G + G^T),
// F_h gains sigma [-p n + tau n] A (sigma = +1 outer, -1 inner probe).
__global__ void __launch_bounds__(IB_PROBE_THREADS) k_adj_probes(
    const MemberDev* __restrict__ mem, const uint8_t* __restrict__ tag, const int* __restrict__ v_cap,
    const CapsuleDev* __restrict__ caps, const double* __restrict__ x, const float* __restrict__ nrm,
    const float* __restrict__ area, const float4* __restrict__ tape, const float4* __restrict__ tape_F, AdjCap a,
    int n_verts) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = t & (GL - 1);
    const int sid = t / GL;
    const int l = min(sid >> 1, n_verts - 1);
    const int s = 1 + (sid & 1);
    const int ax = min(r, 2);
    const float na = nrm[3 * l + ax];
    const double xa = x[3 * l + ax];
    const CapsuleDev& C = caps[v_cap[l]];
    const bool valid = (sid >> 1) < n_verts && !C.rigid;
    const unsigned mask = __ballot_sync(FULL, valid);
    if (!valid) return;
    const MemberDev& d = mem[C.member];
    const double sg = s == 1 ? 1.2 : -1.2;
    const float sigma = s == 1 ? 1.f : -1.f;
    MlsG M;
    float xh, xl, ph, pl;   // the forward probe point, formed as the forward kernel forms it
    split_of(xa, xh, xl);
    probe_of(xh, xl, __fmul_rn(s == 1 ? 1.2f : -1.2f, na), ph, pl);
    mls_build_g<4, PROBE_FAST32>(d, tag, ph, pl, r, mask, M);
    float4 q[GS];
    int node[GS];
#pragma unroll
    for (int j = 0; j < GS; ++j) {
        const int k = r + GL * j;
        node[j] = -1;
        q[j] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (k < 27 && M.W[j] > 0.f) {
            node[j] = mls_node_g(d, M, k);
            q[j] = node_macro(d, tag, tape, tape_F, node[j]);
        }
    }
    // forward: rho_P and G[c][jj] = d u_c / d x_jj at the probe
    float acc[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
#pragma unroll
    for (int j = 0; j < GS; ++j) {
        const int k = r + GL * j;
        if (k >= 27) continue;
        const float p = mls_row_g(M, 0, j, k), g0 = mls_row_g(M, 1, j, k), g1 = mls_row_g(M, 2, j, k),
                    g2 = mls_row_g(M, 3, j, k);
        acc[0] += p * q[j].x;
        acc[1] += g0 * q[j].y; acc[2] += g1 * q[j].y; acc[3] += g2 * q[j].y;
        acc[4] += g0 * q[j].z; acc[5] += g1 * q[j].z; acc[6] += g2 * q[j].z;
        acc[7] += g0 * q[j].w; acc[8] += g1 * q[j].w; acc[9] += g2 * q[j].w;
    }
#pragma unroll
    for (int i = 0; i < 10; ++i) acc[i] = group_sum(acc[i], mask);
    const float rP = acc[0], nu = d.nu;
    const float G[3][3] = {{acc[1], acc[2], acc[3]}, {acc[4], acc[5], acc[6]}, {acc[7], acc[8], acc[9]}};
    const float4 lF4 = a.lF[l];
    const float lF[3] = {lF4.x, lF4.y, lF4.z};
    const float n3[3] = {nrm[3 * l], nrm[3 * l + 1], nrm[3 * l + 2]};
    const float A = area[l];
    const float p = rP * (1.f / 3.f);
    float S[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int jj = 0; jj < 3; ++jj) S[i][jj] = G[i][jj] + G[jj][i];
    // direct terms of n and A, and the adjoints of p and tau
    float ln[3], lAd = 0.f, nlF = 0.f;
#pragma unroll
    for (int i = 0; i < 3; ++i) nlF += n3[i] * lF[i];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        float tl = 0.f, tn = 0.f;
#pragma unroll
        for (int jj = 0; jj < 3; ++jj) {
            tl += rP * nu * S[i][jj] * lF[jj];
            tn += rP * nu * S[i][jj] * n3[jj];
        }
        ln[i] = sigma * A * (-p * lF[i] + tl);
        lAd += sigma * lF[i] * (-p * n3[i] + tn);
    }
    const float lp = -sigma * A * nlF;
    // lambda_tau_ij = sigma A lF_i n_j
    float ltS = 0.f;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int jj = 0; jj < 3; ++jj) ltS += lF[i] * n3[jj] * S[i][jj];
    const float lrP = lp * (1.f / 3.f) + nu * sigma * A * ltS;
    float lG[3][3];   // lambda of d u_c / d x_jj
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int jj = 0; jj < 3; ++jj) lG[c][jj] = rP * nu * sigma * A * (lF[c] * n3[jj] + lF[jj] * n3[c]);
    // support nodes: lambda of (rho_k, u*_k) and the row weights of the MLS product
    float lam[4][GS];
#pragma unroll
    for (int j = 0; j < GS; ++j) {
        const int k = r + GL * j;
        lam[0][j] = lam[1][j] = lam[2][j] = lam[3][j] = 0.f;
        if (k >= 27 || node[j] < 0) continue;
        float lux = 0.f, luy = 0.f, luz = 0.f;
        const float ph = mls_row_g(M, 0, j, k);
        const float ps[3] = {mls_row_g(M, 1, j, k), mls_row_g(M, 2, j, k), mls_row_g(M, 3, j, k)};
        const float lr = ph * lrP;
#pragma unroll
        for (int jj = 0; jj < 3; ++jj) {
            lux += ps[jj] * lG[0][jj];
            luy += ps[jj] * lG[1][jj];
            luz += ps[jj] * lG[2][jj];
        }
        lam[0][j] = lrP * q[j].x;
#pragma unroll
        for (int jj = 0; jj < 3; ++jj)
            lam[1 + jj][j] = lG[0][jj] * q[j].y + lG[1][jj] * q[j].z + lG[2][jj] * q[j].w;
        add4(a.lmac + d.node_off + node[j], lr, lux, luy, luz);
    }
    const f3 lP = mls_vjp_g<4>(M, lam, r, mask);
    if (r == 0) {
        const float sgf = (float)sg;
        add4(a.lx + l, lP.x, lP.y, lP.z);
        add4(a.ln + l, ln[0] + sgf * lP.x, ln[1] + sgf * lP.y, ln[2] + sgf * lP.z);
        atomicAdd(a.lA + l, lAd);
    }
}

// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(IB_MARKER_THREADS) k_adj_markers(
    const MemberDev* __restrict__ mem, const uint8_t* __restrict__ tag, const int* __restrict__ v_cap,
    const CapsuleDev* __restrict__ caps, const CapsuleSums* __restrict__ sums, const double* __restrict__ x,
    const double* __restrict__ vel, const float* __restrict__ nrm, const float* __restrict__ area,
    const float4* __restrict__ tape, const float4* __restrict__ tape_F, AdjCap a, int n_verts) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = t & (GL - 1);
    const int l = min(t / GL, n_verts - 1);
    const int ax = min(r, 2);
    const double P = x[3 * l + ax];
    const float Vb = (float)vel[3 * l + ax];
    const int cap = v_cap[l];
    const CapsuleDev& C = caps[cap];
    const bool valid = t / GL < n_verts && !C.rigid;
    const unsigned mask = __ballot_sync(FULL, valid);
    if (!valid) return;
    const MemberDev& d = mem[C.member];
    MlsG M;
    float Ph, Pl;
    split_of(P, Ph, Pl);
    mls_build_g<4, MARKER_FAST32>(d, tag, Ph, Pl, r, mask, M);
    float ph[GS];
    float4 q[GS], lf[GS];
    int node[GS];
#pragma unroll
    for (int j = 0; j < GS; ++j) {
        const int k = r + GL * j;
        ph[j] = k >= 27 ? 0.f : mls_row_g(M, 0, j, k);
        node[j] = -1;
        q[j] = lf[j] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (ph[j] != 0.f) {
            node[j] = mls_node_g(d, M, k);
            q[j] = node_macro(d, tag, tape, tape_F, node[j]);
            // the forward spreads onto fluid nodes only
            if (q[j].x > 0.f && !(tag[d.node_off + node[j]] & TAG_SOLID)) lf[j] = a.lfib[d.node_off + node[j]];
        }
    }
    float Ux = 0.f, Uy = 0.f, Uz = 0.f, Lx = 0.f, Ly = 0.f, Lz = 0.f;
#pragma unroll
    for (int j = 0; j < GS; ++j) {
        Ux += ph[j] * q[j].y; Uy += ph[j] * q[j].z; Uz += ph[j] * q[j].w;
        Lx += ph[j] * lf[j].x; Ly += ph[j] * lf[j].y; Lz += ph[j] * lf[j].z;
    }
    Ux = group_sum(Ux, mask); Uy = group_sum(Uy, mask); Uz = group_sum(Uz, mask);
    Lx = group_sum(Lx, mask); Ly = group_sum(Ly, mask); Lz = group_sum(Lz, mask);
    const float Fx = __shfl_sync(mask, Vb, 0, GL) - Ux, Fy = __shfl_sync(mask, Vb, 1, GL) - Uy,
                Fz = __shfl_sync(mask, Vb, 2, GL) - Uz;
    const float A = area[l];
    const float lFx = A * Lx, lFy = A * Ly, lFz = A * Lz;   // lambda of F_l through the spreading
    const float4 lU4 = a.lU[l];
    const float lUx = lU4.x - lFx, lUy = lU4.y - lFy, lUz = lU4.z - lFz;
    float lam[1][GS];
    float lAs = 0.f;
#pragma unroll
    for (int j = 0; j < GS; ++j) {
        lam[0][j] = 0.f;
        if (node[j] < 0) continue;
        const float fl = Fx * lf[j].x + Fy * lf[j].y + Fz * lf[j].z;
        lAs += ph[j] * fl;
        lam[0][j] = A * fl + lUx * q[j].y + lUy * q[j].z + lUz * q[j].w;
        add4(a.lmac + d.node_off + node[j], 0.f, ph[j] * lUx, ph[j] * lUy, ph[j] * lUz);
    }
    lAs = group_sum(lAs, mask);
    const f3 lP = mls_vjp_g<1>(M, lam, r, mask);
    double lVp = 0.0;
    if (r == 0) {
        a.lv[l] = make_float4(lFx, lFy, lFz, 0.f);
        add4(a.lx + l, lP.x, lP.y, lP.z);
        // volume penalty k_v (1 - V/V0) A n (Eq. volFor, restoring sign)
        const float kvf = (float)(C.kv * (1.0 - sums[cap].V * C.inv_V0));
        const float4 t4 = a.lF[l];
        const float nx = nrm[3 * l], ny = nrm[3 * l + 1], nz = nrm[3 * l + 2];
        const float nl = nx * t4.x + ny * t4.y + nz * t4.z;
        add4(a.ln + l, kvf * A * t4.x, kvf * A * t4.y, kvf * A * t4.z);
        atomicAdd(a.lA + l, lAs + kvf * nl);
        lVp = -C.kv * C.inv_V0 * (double)A * (double)nl;
    }
    // one atomic per warp when the warp's markers share a capsule
    const unsigned same = __match_any_sync(mask, cap);
    if (same == mask) {
#pragma unroll
        for (int o = 16; o; o >>= 1) lVp += __shfl_xor_sync(mask, lVp, o);
        if ((int)(threadIdx.x & 31) == __ffs(mask) - 1 && lVp != 0.0) atomicAdd(a.lV + cap, lVp);
    } else if (lVp != 0.0) {
        atomicAdd(a.lV + cap, lVp);
    }
}

// ---------------------------------------------------------------------------
// Per triangle (a, b, c) with N = (b - a) x (c - a): S_l gains N/2 and A_l
// gains |N|/6 at each vertex, V gains (a - r0) . N / 6 (r0 the capsule's first
// vertex; the sum of N over a closed surface vanishes, so r0 carries no
// derivative).  n_l = S_l / |S_l| gives lambda_S = (ln - n (n . ln)) / |S|.
__global__ void __launch_bounds__(256) k_adj_geometry(const CapsuleDev* __restrict__ caps, const int* __restrict__ v_cap,
                                                      const float4* __restrict__ xm, const int* __restrict__ tri,
                                                      const float* __restrict__ nrm, AdjCap a, int n_tris) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_tris) return;
    const int ia = tri[3 * t], ib = tri[3 * t + 1], ic = tri[3 * t + 2];
    const int cap = v_cap[ia];
    const CapsuleDev& C = caps[cap];
    if (C.rigid) return;
    const f3 u = mirror_diff(xm, ib, ia), w = mirror_diff(xm, ic, ia), ar = mirror_diff(xm, ia, C.v_begin);
    const f3 N = crs(u, w);
    const float iN = rsqrtf(dot3(N, N));
    const int vs[3] = {ia, ib, ic};
    f3 lS = {0.f, 0.f, 0.f};
    float lAt = 0.f;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const int v = vs[i];
        const f3 n = {nrm[3 * v], nrm[3 * v + 1], nrm[3 * v + 2]};
        const float4 l4 = a.ln[v];
        const f3 ln = {l4.x, l4.y, l4.z};
        const float is = 1.f / a.snorm[v];
        const float nl = dot3(n, ln);
        lS.x += (ln.x - n.x * nl) * is;
        lS.y += (ln.y - n.y * nl) * is;
        lS.z += (ln.z - n.z * nl) * is;
        lAt += a.lA[v];
    }
    const float lv6 = (float)(a.lV[cap] * (1.0 / 6.0));
    const float ca = lAt * (1.f / 6.f) * iN;
    const f3 lN = {0.5f * lS.x + ca * N.x + lv6 * ar.x, 0.5f * lS.y + ca * N.y + lv6 * ar.y,
                   0.5f * lS.z + ca * N.z + lv6 * ar.z};
    const f3 lu = crs(w, lN), lw = crs(lN, u);
    add4(a.lx + ib, lu.x, lu.y, lu.z);
    add4(a.lx + ic, lw.x, lw.y, lw.z);
    add4(a.lx + ia, -lu.x - lw.x + lv6 * N.x, -lu.y - lw.y + lv6 * N.y, -lu.z - lw.z + lv6 * N.z);
}

// ---------------------------------------------------------------------------
// lam_out(k, n) += lambda_rho + (e_k - u*) . lambda_u* / rho at every node of
// the capsules' vertex boxes grown by SHELL_MARGIN (every support node lies
// there), then the node's accumulator is cleared.
__global__ void __launch_bounds__(256) k_adj_fold(const MemberDev* __restrict__ mem, const CapsuleDev* __restrict__ caps,
                                                  const CapsuleSums* __restrict__ sums, const uint8_t* __restrict__ tag,
                                                  const float4* __restrict__ tape, const float4* __restrict__ tape_F,
                                                  float4* __restrict__ lmac, float* __restrict__ lam, size_t LS,
                                                  int n_caps) {
    for (int c = 0; c < n_caps; ++c) {
        const MemberDev& d = mem[caps[c].member];
        const int dims[3] = {d.nx, d.ny, d.nz};
        int lo[3], ext[3];
        bool empty = false;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            int l = sums[c].box_lo[k] - SHELL_MARGIN, h = sums[c].box_hi[k] + SHELL_MARGIN;
            if ((d.per >> k) & 1) {
                h = min(h, l + dims[k] - 1);
            } else {
                l = max(l, 0);
                h = min(h, dims[k] - 1);
            }
            lo[k] = l;
            ext[k] = h - l + 1;
            empty = empty || ext[k] <= 0;
        }
        if (empty) continue;
        const long long total = (long long)ext[0] * ext[1] * ext[2];
        for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
             i += (long long)gridDim.x * blockDim.x) {
            int cx = lo[0] + (int)(i % ext[0]);
            int cy = lo[1] + (int)((i / ext[0]) % ext[1]);
            int cz = lo[2] + (int)(i / ((long long)ext[0] * ext[1]));
            if (d.per & 1) cx = ((cx % d.nx) + d.nx) % d.nx;
            if (d.per & 2) cy = ((cy % d.ny) + d.ny) % d.ny;
            if (d.per & 4) cz = ((cz % d.nz) + d.nz) % d.nz;
            const int n = (cx + d.px) + d.NX * ((cy + d.py) + d.NY * (cz + d.pz));
            const long long gn = d.node_off + n;
            const float4 m = lmac[gn];
            if (m.x == 0.f && m.y == 0.f && m.z == 0.f && m.w == 0.f) continue;
            lmac[gn] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (tag[gn] & TAG_SOLID) continue;
            const float4 q = tape_macro(d, tape, tape_F, n);
            const float ir = 1.f / q.x;
            const float base = m.x - (q.y * m.y + q.z * m.z + q.w * m.w) * ir;
#pragma unroll
            for (int k = 0; k < Q; ++k)
                lam[k * LS + gn] += base + (ex(k) * m.y + ey(k) * m.z + ez(k) * m.w) * ir;
        }
    }
}

// ---------------------------------------------------------------------------
// launches
// ---------------------------------------------------------------------------
cudaError_t launch_adj_capsules(const DevState& d, const AdjCapPtrs& p, const float4* tape_rhou, const float4* tape_F,
                                const double* vel_t, float* lam, size_t LS, cudaStream_t s) {
    if (d.n_verts == 0) return cudaSuccess;
    AdjCap a{p.lx, p.lxp, p.lv, p.lU, p.lF, p.ln, p.lA, p.snorm, p.lV, p.lfib, p.lmac, p.acc_ca};
    const int nv = d.n_verts;
    k_adj_verlet<<<(nv + 255) / 256, 256, 0, s>>>(d.caps, d.v_cap, a, nv);
    if (d.n_edges > 0)
        k_adj_hinges<<<(d.n_edges + 255) / 256, 256, 0, s>>>(d.hinge, d.e_cap, d.caps, d.xm, d.l0, d.ks, d.th0, d.kb, a,
                                                             d.n_edges);
    const long long pt = 2LL * GL * nv;
    k_adj_probes<<<(unsigned)((pt + IB_PROBE_THREADS - 1) / IB_PROBE_THREADS), IB_PROBE_THREADS, 0, s>>>(
        d.mem, d.tag, d.v_cap, d.caps, d.x, d.nrm, d.area, tape_rhou, tape_F, a, nv);
    const long long mt = (long long)GL * nv;
    k_adj_markers<<<(unsigned)((mt + IB_MARKER_THREADS - 1) / IB_MARKER_THREADS), IB_MARKER_THREADS, 0, s>>>(
        d.mem, d.tag, d.v_cap, d.caps, d.sums, d.x, vel_t, d.nrm, d.area, tape_rhou, tape_F, a, nv);
    k_adj_geometry<<<(d.n_tris + 255) / 256, 256, 0, s>>>(d.caps, d.v_cap, d.xm, d.tri, d.nrm, a, d.n_tris);
    k_adj_fold<<<4 * (d.n_sm > 0 ? d.n_sm : 148), 256, 0, s>>>(d.mem, d.caps, d.sums, d.tag, tape_rhou, tape_F, p.lmac,
                                                               lam, LS, d.n_caps);
    return cudaGetLastError();
}

cudaError_t launch_adj_geometry(const DevState& d, double* lV, float* snorm, cudaStream_t s) {
    if (d.n_caps == 0) return cudaSuccess;
    k_adj_geo_reset<<<1, 128, 0, s>>>(d.sums, lV, d.n_caps);
    return launch_geometry_snorm(d, snorm, s);
}

}  // namespace ibl
