// Discrete adjoint of the lattice step (Eq. evoleq collide + stream, Eq.
// bbouzidi wall links, Eq. extbound faces) for lattices without capsules:
// the reverse sweep that carries lambda = dJ/df from the final step back to
// the first, accumulating the derivatives of J with respect to the inlet
// velocity scale and to the junction radius (through the link distances q).
//
// One reverse step t, with lambda the adjoint of the populations after step t:
//   1. faces^T : at every face node, the populations the face rule wrote are
//                replaced by their contributions to the ones it read;
//   2. links^T : every wall link scatters lambda of the population it wrote
//                onto the (up to) three post-collision values it read, each
//                added (atomically) to the lambda entry that the pull of
//                step 3 reads for that value: lambda*_j(p) is found at
//                (j, p + e_j), a solid entry or the entry of the population
//                p streamed to;
//   3. stream^T + collide^T : every fluid node pulls lambda*_i from
//                (i, n + e_i) and applies the transposed collision Jacobian
//                at its (rho, u) of step t; the solid entries holding link
//                terms are then cleared for the buffer's next use.
// The (rho, u) of every node, d(value)/dq of every link and rho of every face
// node come from a tape written while the forward steps are recomputed from a
// checkpoint.
#include "lbm_device.cuh"

namespace ibl {

constexpr unsigned FULLMASK = 0xffffffffu;

__device__ __forceinline__ void block_add_d(double v, double* out) {
    __shared__ double red[32];
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(FULLMASK, v, o);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) red[w] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        double t = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
#pragma unroll
        for (int o = 16; o; o >>= 1) t += __shfl_xor_sync(FULLMASK, t, o);
        if (lane == 0 && t != 0.0) atomicAdd(out, t);
    }
}

// J = sum over the fluid nodes of the box of d . u with u = (sum g e + F/2)/rho,
// and lambda_i = dJ/dg_i = d . (e_i - u) / rho there (zero elsewhere; the
// buffer is cleared before the launch).
__global__ void __launch_bounds__(256) k_adj_objective(const MemberDev* __restrict__ mem, const float* __restrict__ f,
                                                       const uint8_t* __restrict__ tag, int parity, int3 lo, int3 hi,
                                                       double dx, double dy, double dz, float* __restrict__ lam,
                                                       size_t LS, double* __restrict__ J) {
    const MemberDev& d = mem[0];
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    double contrib = 0.0;
    if (n < d.N && !(tag[n] & TAG_SOLID)) {
        int X, Y, Z;
        node_coords(d, n, X, Y, Z);
        const int x = X - d.px, y = Y - d.py, z = Z - d.pz;
        if (x >= lo.x && x < hi.x && y >= lo.y && y < hi.y && z >= lo.z && z < hi.z) {
            float g[Q];
            load_pre<float>(d, f + d.f_off, n, X, Y, Z, parity, g);
            float rho, ux, uy, uz;
            moments_of(g, rho, ux, uy, uz);
            const float ir = __frcp_rn(rho);
            ux += 0.5f * d.F[0] * ir;
            uy += 0.5f * d.F[1] * ir;
            uz += 0.5f * d.F[2] * ir;
            contrib = dx * ux + dy * uy + dz * uz;
            const float du = (float)(dx * ux + dy * uy + dz * uz);
#pragma unroll
            for (int k = 0; k < Q; ++k)
                lam[k * LS + n] = ((float)dx * ex(k) + (float)dy * ey(k) + (float)dz * ez(k) - du) * ir;
        }
    }
    block_add_d(contrib, J);
}

// faces^T, in place.  With c_j = 1 (e_j.n = 0), 2 (e_j.n > 0), 0 (e_j.n < 0)
// and D = 1 + u_w.n, the face rule writes for every k with e_k.n < 0,
// t = e_k + n, o = opp(k):
//   velocity face: v_k = g_o + rho a_k - (1/2) sum_{e_j.n=0} g_j (e_j.t),
//                  rho = (1 + sum c_j g_j) / D,
//                  a_k = -u_n/3 (t = 0) or -u_n/6 + u_t/2 (t != 0)
//   pressure face: v_k = g_o - (1 + sum c_j g_j) / (3 or 6) - (1/2) sum_{e_j.n=0} g_j (e_j.t)
// so dv_k/dg_j = delta_jo + (a_k / D or -1/3, -1/6) c_j - (1/2)[e_j.n = 0](e_j.t).
// Scaling the inlet velocities by (1 + s) gives dv_k/ds = a_k rho / D.
__global__ void __launch_bounds__(256) k_adj_faces(const MemberDev* __restrict__ mem,
                                                   const uint32_t* __restrict__ fc_node,
                                                   const uint32_t* __restrict__ fc_meta,
                                                   const float* __restrict__ face_vel,
                                                   const float* __restrict__ tape_rho, float* __restrict__ lam,
                                                   size_t LS, int n_face_nodes, double* __restrict__ grad_s) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double ds = 0.0;
    if (i < n_face_nodes) {
        const MemberDev& d = mem[0];
        const int fc = (int)(fc_meta[i] & 7u);
        const int n = (int)fc_node[i];
        const int nx = fc == 0 ? -1 : (fc == 1 ? 1 : 0);
        const int ny = fc == 2 ? -1 : (fc == 3 ? 1 : 0);
        const int nz = fc == 4 ? -1 : (fc == 5 ? 1 : 0);
        const bool vel = d.face_kind[fc] == FACE_VELOCITY;
        float uwx = 0.f, uwy = 0.f, uwz = 0.f;
        if (vel) {
            int X, Y, Z;
            node_coords(d, n, X, Y, Z);
            const float* u = face_vel + 3 * (d.face_off[fc] + face_index(d, fc, X, Y, Z));
            uwx = u[0]; uwy = u[1]; uwz = u[2];
        }
        const float un = uwx * nx + uwy * ny + uwz * nz;
        const float iD = 1.f / (1.f + un);
        float l[Q], out[Q];
#pragma unroll
        for (int k = 0; k < Q; ++k) {
            l[k] = lam[k * LS + n];
            out[k] = (ex(k) * nx + ey(k) * ny + ez(k) * nz) < 0 ? 0.f : l[k];
        }
        const float rho = vel ? tape_rho[i] : 0.f;
#pragma unroll
        for (int k = 0; k < Q; ++k) {
            if (ex(k) * nx + ey(k) * ny + ez(k) * nz >= 0) continue;
            const int tx = ex(k) + nx, ty = ey(k) + ny, tz = ez(k) + nz;
            const bool axial = tx == 0 && ty == 0 && tz == 0;
            const float ut = uwx * tx + uwy * ty + uwz * tz;
            const float a = axial ? -un * (1.f / 3.f) : (-un * (1.f / 6.f) + 0.5f * ut);
            const float crho = vel ? a * iD : (axial ? -1.f / 3.f : -1.f / 6.f);
            const float lk = l[k];
            out[opp(k)] += lk;
#pragma unroll
            for (int j = 0; j < Q; ++j) {
                const int en = ex(j) * nx + ey(j) * ny + ez(j) * nz;
                const float c = en == 0 ? 1.f : (en > 0 ? 2.f : 0.f);
                float coef = crho * c;
                if (en == 0) coef -= 0.5f * (float)(ex(j) * tx + ey(j) * ty + ez(j) * tz);
                out[j] += coef * lk;
            }
            if (vel) ds += (double)lk * (double)(a * rho * iD);
        }
#pragma unroll
        for (int k = 0; k < Q; ++k) lam[k * LS + n] = out[k];
    }
    block_add_d(ds, grad_s);
}

// links^T: the value the wall rule wrote at (opp(i), x_b) is a combination of
// f*_i(x_b), f*_i(x_b - e_i), f*_i(x_b - 2 e_i), f*_opp(i)(x_b), f*_opp(i)(x_b - e_i)
// with the coefficients of the forward rule; dJ/dr_j gains
// lambda * (d value / dq) * (dq / dr_j).  No entry that a link reads is
// written by another link (a link's reads and writes sit on opposite sides of
// its wall), so the scatter runs in place on lambda.
__global__ void __launch_bounds__(256) k_adj_links(const MemberDev* __restrict__ mem,
                                                   const uint32_t* __restrict__ l_node,
                                                   const uint32_t* __restrict__ l_meta, const float* __restrict__ l_q,
                                                   const float* __restrict__ l_dq, const float* __restrict__ tape_dvdq,
                                                   float* __restrict__ lam, size_t LS, int n_links,
                                                   double* __restrict__ grad_q) {
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    double dqs = 0.0;
    if (l < n_links) {
        const MemberDev& d = mem[0];
        const uint32_t meta = l_meta[l];
        const int i = (int)(meta & 31u), ib = opp(i);
        const bool ok1 = meta & 32u, ok2 = meta & 64u;
        const int xb = (int)l_node[l];
        const float lv = lam[ib * LS + xb];
        if (lv != 0.f) {
            const float q = l_q[l];
            int X, Y, Z;
            node_coords(d, xb, X, Y, Z);
            const bool px = d.per & 1, py = d.per & 2, pz = d.per & 4;
            const int exi = ex(i), eyi = ey(i), ezi = ez(i);
            const int s0 = nbc(X, exi, d.NX, px) + d.NX * (nbc(Y, eyi, d.NY, py) + d.NY * nbc(Z, ezi, d.NZ, pz));
            const int X1 = nbc(X, -exi, d.NX, px), Y1 = nbc(Y, -eyi, d.NY, py), Z1 = nbc(Z, -ezi, d.NZ, pz);
            const int m1 = X1 + d.NX * (Y1 + d.NY * Z1);
            float* li = lam + i * LS;    // lambda*_i(p) sits at (i, p + e_i)
            float* lb = lam + ib * LS;   // lambda*_ib(p) sits at (ib, p - e_i)
            if (q < 0.5f) {
                if (ok1 && ok2) {
                    atomicAdd(li + s0, q * (2.f * q + 1.f) * lv);
                    atomicAdd(li + xb, (1.f - 4.f * q * q) * lv);
                    atomicAdd(li + m1, -q * (1.f - 2.f * q) * lv);
                } else if (ok1) {
                    atomicAdd(li + s0, 2.f * q * lv);
                    atomicAdd(li + xb, (1.f - 2.f * q) * lv);
                } else {
                    atomicAdd(li + s0, lv);
                }
            } else {
                if (ok1) {
                    const int m2 = nbc(X1, -exi, d.NX, px) +
                                   d.NX * (nbc(Y1, -eyi, d.NY, py) + d.NY * nbc(Z1, -ezi, d.NZ, pz));
                    atomicAdd(li + s0, lv / (q * (2.f * q + 1.f)));
                    atomicAdd(lb + m1, (2.f * q - 1.f) / q * lv);
                    atomicAdd(lb + m2, (1.f - 2.f * q) / (1.f + 2.f * q) * lv);
                } else {
                    atomicAdd(li + s0, lv / (2.f * q));
                    atomicAdd(lb + m1, (2.f * q - 1.f) / (2.f * q) * lv);
                }
            }
            dqs = (double)lv * (double)tape_dvdq[l] * (double)l_dq[l];
        }
    }
    block_add_d(dqs, grad_q);
}

// stream^T + links + collide^T at every fluid node.  With omega = 1/tau,
// guo = 1 - omega/2, the collision f*_j = f_j - omega (f_j - f^eq_j(rho, u))
// + G_j(u) has d rho/d f_i = 1 and d u/d f_i = (e_i - u)/rho, so
//   lambda_i = (1 - omega) lambda*_i + omega A + B . (e_i - u) / rho,
//   A = sum_j lambda*_j w_j (1 + 3 e_j.u + 9/2 (e_j.u)^2 - 3/2 u^2),
//   B = sum_j lambda*_j [omega w_j rho (3 e_j + 9 (e_j.u) e_j - 3 u)
//                        + guo w_j (9 (e_j.F) e_j - 3 F)].
// Entries at solid nodes hold only link terms (zero otherwise), so every
// neighbour is pulled without a tag test; k_adj_clear zeroes the link terms
// once they are consumed.  Work list: the aligned 32-node runs that hold a
// fluid node, one warp per run; interior runs address neighbours by constant
// offsets, border runs (periodic wrap planes) by coordinates.
// With capsules, F = F_body + f_ib(n) varies per node: the IB part comes from
// a tape (w = 1 where the node received spreading), and at those nodes the
// kernel also returns lambda_F = d f* / d F . lambda*: u depends on F through
// rho u = sum f e + F/2, and the Guo term directly, so
//   lambda_F = B / (2 rho) + guo sum_j lambda*_j w_j [3 (e_j - u) + 9 (e_j.u) e_j].
template <bool BORDER>
__global__ void __launch_bounds__(256) k_adj_step(const __grid_constant__ MemberDev d, const uint8_t* __restrict__ tag,
                                                  const uint32_t* __restrict__ segs, int n_segs,
                                                  const float4* __restrict__ tape, const float* __restrict__ lam_in,
                                                  float* __restrict__ lam_out, size_t LS,
                                                  const float4* __restrict__ tape_F, float4* __restrict__ lam_fib) {
    const int si = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (si >= n_segs) return;
    const int n = (int)(segs[si] << 5) + (int)(threadIdx.x & 31);
    if (n >= d.N || (tag[n] & TAG_SOLID)) return;
    float ls[Q];
    if (BORDER) {
        int X, Y, Z;
        node_coords(d, n, X, Y, Z);
        const Nbr b = neighbours(d, X, Y, Z);
#pragma unroll
        for (int k = 0; k < Q; ++k)
            ls[k] = lam_in[k * LS + b.xs[1 + ex(k)] + d.NX * (b.ys[1 + ey(k)] + d.NY * b.zs[1 + ez(k)])];
    } else {
#pragma unroll
        for (int k = 0; k < Q; ++k) ls[k] = lam_in[k * LS + (n + lin_off(d, k))];
    }
    const float4 t = tape[n];
    const float rho = t.x, ux = t.y, uy = t.z, uz = t.w;
    float Fx = d.F[0], Fy = d.F[1], Fz = d.F[2];
    bool ibn = false;
    if (tape_F) {
        const float4 fi = tape_F[n];
        ibn = fi.w != 0.f;
        Fx += fi.x; Fy += fi.y; Fz += fi.z;
    }
    const float om = d.omega, guo = d.guo;
    const float usq = 1.5f * (ux * ux + uy * uy + uz * uz);
    const float orho = om * rho;
    // A and B summed by opposite pairs (k, kb): e.u and e.F change sign
    // between the two, so with dw = w_k l_k - w_kb l_kb and sw = w_k l_k +
    // w_kb l_kb the pair adds 3 (e.u) dw + 9/2 (e.u)^2 sw to A (beyond
    // (1 - 3/2 u^2) times the sum of all w l) and e_k [3 om rho dw +
    // 9 (om rho e.u + guo e.F) sw] to B (beyond -(3 om rho u + 3 guo F)
    // times the same sum).
    float W = wgt(0) * ls[0];
    float A = 0.f, Bx = 0.f, By = 0.f, Bz = 0.f, Cx = 0.f, Cy = 0.f, Cz = 0.f;
#pragma unroll
    for (int k = 1; k < Q; ++k) {
        if (opp(k) < k) continue;
        const int kb = opp(k);
        const float eu = ex(k) * ux + ey(k) * uy + ez(k) * uz;
        const float eF = ex(k) * Fx + ey(k) * Fy + ez(k) * Fz;
        const float dw = wgt(k) * (ls[k] - ls[kb]), sw = wgt(k) * (ls[k] + ls[kb]);
        W += sw;
        A += eu * (3.f * dw + 4.5f * eu * sw);
        const float c = 3.f * orho * dw + 9.f * (orho * eu + guo * eF) * sw;
        if (ex(k)) Bx += ex(k) * c;
        if (ey(k)) By += ey(k) * c;
        if (ez(k)) Bz += ez(k) * c;
        if (ibn) {
            // sum_j lambda*_j w_j [3 e_j + 9 (e_j.u) e_j] by pairs
            const float cc = 3.f * dw + 9.f * eu * sw;
            if (ex(k)) Cx += ex(k) * cc;
            if (ey(k)) Cy += ey(k) * cc;
            if (ez(k)) Cz += ez(k) * cc;
        }
    }
    A += W * (1.f - usq);
    Bx -= W * (3.f * orho * ux + 3.f * guo * Fx);
    By -= W * (3.f * orho * uy + 3.f * guo * Fy);
    Bz -= W * (3.f * orho * uz + 3.f * guo * Fz);
    const float ir = 1.f / rho;
    if (ibn) {
        const float h = 0.5f * ir;
        lam_fib[n] = make_float4(Bx * h + guo * (Cx - 3.f * ux * W), By * h + guo * (Cy - 3.f * uy * W),
                                 Bz * h + guo * (Cz - 3.f * uz * W), 0.f);
    }
    const float Bu = Bx * ux + By * uy + Bz * uz;
    const float base = om * A - Bu * ir, keep = 1.f - om;
    lam_out[n] = keep * ls[0] + base;
#pragma unroll
    for (int k = 1; k < Q; ++k) {
        if (opp(k) < k) continue;
        const int kb = opp(k);
        const float be = (Bx * ex(k) + By * ey(k) + Bz * ez(k)) * ir;
        lam_out[k * LS + n] = keep * ls[k] + base + be;
        lam_out[kb * LS + n] = keep * ls[kb] + base - be;
    }
}

// The solid entries a link wrote in links^T, cleared after k_adj_step has
// pulled them (its fluid entries are overwritten when the buffer next
// receives a step's output).
__global__ void __launch_bounds__(256) k_adj_clear(const __grid_constant__ MemberDev d,
                                                   const uint8_t* __restrict__ tag,
                                                   const uint32_t* __restrict__ l_node,
                                                   const uint32_t* __restrict__ l_meta, float* __restrict__ lam,
                                                   size_t LS, int n_links) {
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= n_links) return;
    const uint32_t meta = l_meta[l];
    const int i = (int)(meta & 31u), ib = opp(i);
    const int xb = (int)l_node[l];
    int X, Y, Z;
    node_coords(d, xb, X, Y, Z);
    const bool px = d.per & 1, py = d.per & 2, pz = d.per & 4;
    const int exi = ex(i), eyi = ey(i), ezi = ez(i);
    const int s0 = nbc(X, exi, d.NX, px) + d.NX * (nbc(Y, eyi, d.NY, py) + d.NY * nbc(Z, ezi, d.NZ, pz));
    const int X1 = nbc(X, -exi, d.NX, px), Y1 = nbc(Y, -eyi, d.NY, py), Z1 = nbc(Z, -ezi, d.NZ, pz);
    const int m1 = X1 + d.NX * (Y1 + d.NY * Z1);                // in range: x_b is an interior node
    lam[i * LS + s0] = 0.f;                                     // s0 is solid
    if (tag[m1] & TAG_SOLID) {
        lam[ib * LS + m1] = 0.f;
    } else {                                                    // m1 fluid: m2 is in range too
        const int m2 = nbc(X1, -exi, d.NX, px) + d.NX * (nbc(Y1, -eyi, d.NY, py) + d.NY * nbc(Z1, -ezi, d.NZ, pz));
        if (tag[m2] & TAG_SOLID) lam[ib * LS + m2] = 0.f;
    }
}

cudaError_t launch_adj_objective(const DevState& d, int parity, const int lo[3], const int hi[3], const double w[3],
                                 float* lam, size_t LS, double* J, cudaStream_t s) {
    const int N = d.h_mem[0].N;
    k_adj_objective<<<(N + 255) / 256, 256, 0, s>>>(d.mem, (const float*)d.f, d.tag, parity,
                                                    make_int3(lo[0], lo[1], lo[2]), make_int3(hi[0], hi[1], hi[2]),
                                                    w[0], w[1], w[2], lam, LS, J);
    return cudaGetLastError();
}

cudaError_t launch_adj_step(const DevState& d, const float* tape_rho, const float* tape_dvdq, const float4* tape_rhou,
                            float* lam_in, float* lam_out, size_t LS, double* grad_s, double* grad_q,
                            cudaStream_t s, const float4* tape_F, float4* lam_fib) {
    if (d.n_face_nodes > 0)
        k_adj_faces<<<(d.n_face_nodes + 255) / 256, 256, 0, s>>>(d.mem, d.fc_node, d.fc_meta, d.face_vel, tape_rho,
                                                                 lam_in, LS, d.n_face_nodes, grad_s);
    if (d.n_links > 0)
        k_adj_links<<<(d.n_links + 255) / 256, 256, 0, s>>>(d.mem, d.l_node, d.l_meta, d.l_q, d.l_dq, tape_dvdq,
                                                            lam_in, LS, d.n_links, grad_q);
    const MemberDev& md = d.h_mem[0];
    if (d.n_segs > 0)
        k_adj_step<false><<<(d.n_segs + 7) / 8, 256, 0, s>>>(md, d.tag, d.segs, d.n_segs, tape_rhou, lam_in, lam_out, LS,
                                                             tape_F, lam_fib);
    if (d.n_bsegs > 0)
        k_adj_step<true><<<(d.n_bsegs + 7) / 8, 256, 0, s>>>(md, d.tag, d.bsegs, d.n_bsegs, tape_rhou, lam_in, lam_out,
                                                             LS, tape_F, lam_fib);
    if (d.n_links > 0)
        k_adj_clear<<<(d.n_links + 255) / 256, 256, 0, s>>>(md, d.tag, d.l_node, d.l_meta, lam_in, LS, d.n_links);
    return cudaGetLastError();
}

}  // namespace ibl
