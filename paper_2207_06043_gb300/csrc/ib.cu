// Immersed-boundary and structure kernels: per-capsule geometry, the MLS
// interpolate/force/spread pass with the probe stresses and volume penalty
// (four lanes per stencil), per-hinge stretching + bending, inter-body
// repulsion on a cell list, and the Verlet / Newton-Euler update with the
// damage rule.
#include <climits>

#include "ib_device.cuh"

namespace ibl {



__global__ void __launch_bounds__(256) k_mirror(const double* __restrict__ x, float4* __restrict__ xm, int n_verts) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v < n_verts) mirror_put(xm, v, x[3 * v], x[3 * v + 1], x[3 * v + 2]);
}



// ---------------------------------------------------------------------------
// Per-capsule geometry at x(t), spread over GEO_BLOCKS blocks per capsule:
// per triangle, the area-weighted normal and a third of the area go to its
// vertices (float4 atomics into vacc); the enclosed volume (divergence theorem,
// tetrahedra fanned from the capsule's first vertex, each term in FP32 from
// FP64 differences) is summed in FP64.  Then
// per vertex: A_v = 1/3 sum of adjacent triangle areas, n_v = normalised
// area-weighted sum of adjacent normals, the integer bounding box, and vacc
// is cleared for the next step.  V and the box are reset at the step begin.
// ---------------------------------------------------------------------------
constexpr int GEO_BLOCKS = 16;


__global__ void __launch_bounds__(256) k_geom_tri(const CapsuleDev* __restrict__ caps, CapsuleSums* __restrict__ sums,
                                                  const uint32_t* __restrict__ status, const float4* __restrict__ xm,
                                                  const int* __restrict__ tri, float4* __restrict__ vacc) {
    __shared__ double red[32];
    const int c = blockIdx.x / GEO_BLOCKS, part = blockIdx.x % GEO_BLOCKS;
    const CapsuleDev& C = caps[c];
    if (status[C.member] & STOP) return;
    const int vb = C.v_begin;
    double vol = 0.0;
    for (int t = C.t_begin + part * blockDim.x + threadIdx.x; t < C.t_begin + C.t_count;
         t += GEO_BLOCKS * blockDim.x) {
        const int ia = tri[3 * t], ib = tri[3 * t + 1], ic = tri[3 * t + 2];
        // edges from vertex a
        const f3 u = mirror_diff(xm, ib, ia), w = mirror_diff(xm, ic, ia);
        const float Nx = u.y * w.z - u.z * w.y, Ny = u.z * w.x - u.x * w.z, Nz = u.x * w.y - u.y * w.x;
        // tetrahedron (r0, a, b, c): a . (b x c) / 6 = a . ((b - a) x (c - a)) / 6
        // with a relative to r0 = the first vertex; the term in FP32, the sum
        // in FP64
        const f3 a = mirror_diff(xm, ia, vb);
        vol += (double)(a.x * Nx + a.y * Ny + a.z * Nz);
        const float a3 = sqrtf(Nx * Nx + Ny * Ny + Nz * Nz) * (1.f / 6.f);
        const float4 contrib = make_float4(0.5f * Nx, 0.5f * Ny, 0.5f * Nz, a3);
        atomicAdd(vacc + ia, contrib);   // vector reductions, one per vertex of the triangle
        atomicAdd(vacc + ib, contrib);
        atomicAdd(vacc + ic, contrib);
    }
    const double s = block_sum_d(vol, red);
    if (threadIdx.x == 0) atomicAdd(&sums[c].V, s * (1.0 / 6.0));
}

__global__ void __launch_bounds__(256) k_geom_vtx(const CapsuleDev* __restrict__ caps, const int* __restrict__ v_cap,
                                                  CapsuleSums* __restrict__ sums, const uint32_t* __restrict__ status,
                                                  const float4* __restrict__ xm, float4* __restrict__ vacc,
                                                  float* __restrict__ nrm, float* __restrict__ area, int n_verts,
                                                  float* __restrict__ snorm) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = v < n_verts && !(status[caps[v_cap[min(v, n_verts - 1)]].member] & STOP);
    const int c = live ? v_cap[v] : -1;
    int lo[3] = {INT_MAX, INT_MAX, INT_MAX}, hi[3] = {INT_MIN, INT_MIN, INT_MIN};
    int r2lo = 0x7f800000, r2hi = 0;   // FP32 bits (non-negative: integer order is value order)
    if (live) {
        const float4 a = vacc[v];
        const float inv = rsqrtf(a.x * a.x + a.y * a.y + a.z * a.z);
        if (snorm) snorm[v] = sqrtf(a.x * a.x + a.y * a.y + a.z * a.z);   // |S_l| for the adjoint
        nrm[3 * v] = a.x * inv;
        nrm[3 * v + 1] = a.y * inv;
        nrm[3 * v + 2] = a.z * inv;
        area[v] = a.w;
        vacc[v] = make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 h4 = xm[2 * v], l4 = xm[2 * v + 1];
        const float hv[3] = {h4.x, h4.y, h4.z}, lv[3] = {l4.x, l4.y, l4.z};
        float r2 = 0.f;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            // floor(x) from x = hi + lo (|lo| <= half an ulp of hi): floor(hi),
            // less one when hi is an integer and lo < 0
            const float fh = floorf(hv[k]);
            const float fx = (fh == hv[k] && lv[k] < 0.f) ? fh - 1.f : fh;
            lo[k] = isfinite(hv[k]) ? (int)fmaxf(fminf(fx, 1e9f), -1e9f) : 0;
            hi[k] = lo[k] + 1;
            const float dq = (hv[k] - sums[c].rcf[k]) + lv[k];
            r2 += dq * dq;
        }
        if (r2 >= 0.f && r2 < 1e30f) { r2lo = __float_as_int(r2); r2hi = r2lo; }
        else { r2lo = 0; r2hi = 0x7f800000; }   // not finite: no radial bound
    }
    // lanes of one capsule reduce among themselves, then one lane per capsule
    // and warp updates the box (consecutive vertices share a capsule)
    const unsigned peers = __match_any_sync(FULL, c);
    const int leader = __ffs(peers) - 1;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        lo[k] = __reduce_min_sync(peers, lo[k]);
        hi[k] = __reduce_max_sync(peers, hi[k]);
    }
    r2lo = __reduce_min_sync(peers, r2lo);
    r2hi = __reduce_max_sync(peers, r2hi);
    if (live && (int)(threadIdx.x & 31) == leader) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            atomicMin(&sums[c].box_lo[k], lo[k]);
            atomicMax(&sums[c].box_hi[k], hi[k]);
        }
        atomicMin(&sums[c].r2_lo, r2lo);
        atomicMax(&sums[c].r2_hi, r2hi);
    }
}


// One warp per row (y, z) of a capsule's box, lanes along x over the part of
// the row inside the outer sphere, less the part inside the inner one.
template <typename T, bool LIN>
__device__ __forceinline__ void shell_rows(const MemberDev& d, const T* __restrict__ fm, uint8_t* __restrict__ tag,
                                           float4* __restrict__ macro,
                                           const int lo[3], const int ext[3], bool radial, float r2_out, float r2_in,
                                           float rcx, float rcy, float rcz, int parity) {
    const int lane = threadIdx.x & 31;
    const int nwarps = SHELL_BLOCKS * (int)(blockDim.x >> 5);
    const int rows = ext[1] * ext[2];
    for (int row = (blockIdx.x % SHELL_BLOCKS) * (int)(blockDim.x >> 5) + (int)(threadIdx.x >> 5); row < rows;
         row += nwarps) {
        const int iz = row / ext[1], iy = row - iz * ext[1];
        int cy = lo[1] + iy, cz = lo[2] + iz;
        const float qy = (float)cy - rcy, qz = (float)cz - rcz;
        const float d2 = qy * qy + qz * qz;
        int x0 = lo[0], x1 = lo[0] + ext[0] - 1;
        float hin = -1.f;
        if (radial) {
            if (d2 > r2_out) continue;   // the whole row (uniform over the warp)
            const float hw = sqrtf(r2_out - d2);
            x0 = max(x0, (int)ceilf(rcx - hw));
            x1 = min(x1, (int)floorf(rcx + hw));
            if (r2_in > d2) hin = sqrtf(r2_in - d2);
        }
        if (!LIN) {
            if (d.per & 2) cy = ((cy % d.ny) + d.ny) % d.ny;
            if (d.per & 4) cz = ((cz % d.nz) + d.nz) % d.nz;
        }
        const int Y = cy + d.py, Z = cz + d.pz;
        for (int cx = x0 + lane; cx <= x1; cx += 32) {
            if (fabsf((float)cx - rcx) < hin) continue;
            int wx = cx;
            if (!LIN && (d.per & 1)) wx = ((wx % d.nx) + d.nx) % d.nx;
            const int X = wx + d.px;
            const int node = X + d.NX * (Y + d.NY * Z);
            // a solid node holds the wall's state, rho = 1 and u = 0, stored
            // with rho negated so that the marker stencils know not to spread
            // onto it without a tag gather; the populations' loads are issued
            // beside the tag's, so they do not wait on it.  A fluid node takes
            // the IB flag: the marker stencils spread onto band nodes only,
            // and the lattice step adds the node's f_ib and clears both
            const bool solid = tag[d.node_off + node] & TAG_SOLID;
            if (!solid) tag[d.node_off + node] = TAG_IB;
            float g[Q];
            if (LIN) load_pre_lin<T>(d, fm, node, parity, g);
            else load_pre<T>(d, fm, node, X, Y, Z, parity, g);
            float rho, ux, uy, uz;
            moments_of(g, rho, ux, uy, uz);
            macro[d.node_off + node] = solid ? make_float4(-1.f, 0.f, 0.f, 0.f) : make_float4(rho, ux, uy, uz);
        }
    }
}

// The capsule's box grown by the shell margin (clipped to the box, or at most
// one period on a periodic axis) and its radial band: false if empty.
__device__ __forceinline__ bool shell_box(const MemberDev& d, const CapsuleSums& S, int lo[3], int ext[3],
                                          bool& radial, float& r2_out, float& r2_in) {
    const int dims[3] = {d.nx, d.ny, d.nz};
    bool wide = false;   // a grown box wider than a periodic lattice: no radial test
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        int l = S.box_lo[a] - SHELL_MARGIN, h = S.box_hi[a] + SHELL_MARGIN;
        if ((d.per >> a) & 1) {
            wide = wide || h > l + dims[a] - 1;
            h = min(h, l + dims[a] - 1);
        } else {
            l = max(l, 0);
            h = min(h, dims[a] - 1);
        }
        lo[a] = l;
        ext[a] = h - l + 1;
    }
    if (ext[0] <= 0 || ext[1] <= 0 || ext[2] <= 0) return false;
    // annulus of the vertices about rc, grown by the stencils' reach
    const float rhi = sqrtf(__int_as_float(S.r2_hi)) + SHELL_REACH;
    const float rlo = sqrtf(__int_as_float(S.r2_lo)) - SHELL_REACH;
    radial = !wide && rhi < 1e6f;   // no radial test for a non-finite or over-wide capsule
    r2_out = rhi * rhi;
    r2_in = (radial && rlo > 0.f) ? rlo * rlo : -1.f;
    return true;
}

// fn(x, y, z) for every node of the capsule's shell (user coordinates, wrapped
// on periodic axes), one warp per row as in shell_rows.
template <typename F>
__device__ __forceinline__ void for_shell_nodes(const MemberDev& d, const int lo[3], const int ext[3], bool radial,
                                                float r2_out, float r2_in, float rcx, float rcy, float rcz, F fn) {
    const int lane = threadIdx.x & 31;
    const int nwarps = SHELL_BLOCKS * (int)(blockDim.x >> 5);
    const int rows = ext[1] * ext[2];
    for (int row = (blockIdx.x % SHELL_BLOCKS) * (int)(blockDim.x >> 5) + (int)(threadIdx.x >> 5); row < rows;
         row += nwarps) {
        const int iz = row / ext[1], iy = row - iz * ext[1];
        int cy = lo[1] + iy, cz = lo[2] + iz;
        const float qy = (float)cy - rcy, qz = (float)cz - rcz;
        const float d2 = qy * qy + qz * qz;
        int x0 = lo[0], x1 = lo[0] + ext[0] - 1;
        float hin = -1.f;
        if (radial) {
            if (d2 > r2_out) continue;
            const float hw = sqrtf(r2_out - d2);
            x0 = max(x0, (int)ceilf(rcx - hw));
            x1 = min(x1, (int)floorf(rcx + hw));
            if (r2_in > d2) hin = sqrtf(r2_in - d2);
        }
        if (d.per & 2) cy = ((cy % d.ny) + d.ny) % d.ny;
        if (d.per & 4) cz = ((cz % d.nz) + d.nz) % d.nz;
        for (int cx = x0 + lane; cx <= x1; cx += 32) {
            if (fabsf((float)cx - rcx) < hin) continue;
            int wx = cx;
            if (d.per & 1) wx = ((wx % d.nx) + d.nx) % d.nx;
            fn(wx, cy, cz);
        }
    }
}

// LIN_ONLY: every lattice of the context has no periodic axis and none is a
// slab context's whole view, so only the constant-offset path is compiled,
// in 48 registers with 5 resident blocks per SM instead of 80 and 3.
template <typename T, bool LIN_ONLY>
__global__ void __launch_bounds__(256, LIN_ONLY ? 5 : 3) k_shell(const MemberDev* __restrict__ mem, const T* __restrict__ f,
                                               uint8_t* __restrict__ tag,
                                               const uint32_t* __restrict__ status, const CapsuleDev* __restrict__ caps,
                                               const CapsuleSums* __restrict__ sums, float4* __restrict__ macro,
                                               int parity, float* __restrict__ fib, const int* __restrict__ slab_of,
                                               const int4* __restrict__ slab_tab) {
    const int c = blockIdx.x / SHELL_BLOCKS;
    const CapsuleDev& C = caps[c];
    if (status[C.member] & STOP) return;
    const MemberDev& d = mem[C.member];
    int lo[3], ext[3];
    bool radial;
    float r2_out, r2_in;
    if (!shell_box(d, sums[c], lo, ext, radial, r2_out, r2_in)) return;
    const float rcx = sums[c].rcf[0], rcy = sums[c].rcf[1], rcz = sums[c].rcf[2];
    if (LIN_ONLY) {
        shell_rows<T, true>(d, f + d.f_off, tag, macro, lo, ext, radial, r2_out, r2_in, rcx, rcy, rcz, parity);
        return;
    }
    if (d.slab_view) {
        // the whole lattice of a slab context: each node's populations from the
        // slab that owns it (its neighbours are in that slab's ghost planes);
        // the node's IB force of the previous step is cleared here, as the
        // lattice kernel does for a lattice of its own, and a fluid node
        // takes the IB flag
        for_shell_nodes(d, lo, ext, radial, r2_out, r2_in, rcx, rcy, rcz, [&](int x, int y, int z) {
            const long long nW = d.node_off + (x + d.px) + (long long)d.NX * ((y + d.py) + (long long)d.NY * (z + d.pz));
            const int s = slab_of[x];
            const MemberDev& ds = mem[s];
            const int4 t = slab_tab[s];
            const int X = x - (t.x - t.z) + ds.px, Y = y + ds.py, Z = z + ds.pz;
            const int n = X + ds.NX * (Y + ds.NY * Z);
            const bool solid = tag[nW] & TAG_SOLID;
            float g[Q];
            load_pre<T>(ds, f + ds.f_off, n, X, Y, Z, parity, g);
            float rho, ux, uy, uz;
            moments_of(g, rho, ux, uy, uz);
            macro[nW] = solid ? make_float4(-1.f, 0.f, 0.f, 0.f) : make_float4(rho, ux, uy, uz);
            reinterpret_cast<float4*>(fib)[nW] = make_float4(0.f, 0.f, 0.f, 0.f);
            tag[nW] = solid ? TAG_SOLID : TAG_IB;
        });
        return;
    }
    const T* fm = f + d.f_off;
    // a lattice with no periodic axis reaches every upstream node at a
    // constant offset (the ghost layer absorbs the steps off the box)
    if (d.per == 0)
        shell_rows<T, true>(d, fm, tag, macro, lo, ext, radial, r2_out, r2_in, rcx, rcy, rcz, parity);
    else
        shell_rows<T, false>(d, fm, tag, macro, lo, ext, radial, r2_out, r2_in, rcx, rcy, rcz, parity);
}

// The IB force the markers spread into the whole-lattice member of a slab
// context, copied to every slab that holds the node (its owner and the ghost
// planes of its neighbours), with the node's IB flag, for the slabs' lattice
// step.
__global__ void __launch_bounds__(256) k_fib_scatter(const MemberDev* __restrict__ mem, uint8_t* __restrict__ tag,
                                                      float* __restrict__ fib, const uint32_t* __restrict__ status,
                                                      const CapsuleDev* __restrict__ caps,
                                                      const CapsuleSums* __restrict__ sums,
                                                      const int* __restrict__ slab_of,
                                                      const int4* __restrict__ slab_tab, int n_slabs) {
    const int c = blockIdx.x / SHELL_BLOCKS;
    const CapsuleDev& C = caps[c];
    if (status[C.member] & STOP) return;
    const MemberDev& d = mem[C.member];
    int lo[3], ext[3];
    bool radial;
    float r2_out, r2_in;
    if (!shell_box(d, sums[c], lo, ext, radial, r2_out, r2_in)) return;
    const float rcx = sums[c].rcf[0], rcy = sums[c].rcf[1], rcz = sums[c].rcf[2];
    for_shell_nodes(d, lo, ext, radial, r2_out, r2_in, rcx, rcy, rcz, [&](int x, int y, int z) {
        const long long nW = d.node_off + (x + d.px) + (long long)d.NX * ((y + d.py) + (long long)d.NY * (z + d.pz));
        if (!(tag[nW] & TAG_IB)) return;
        const float4 v = reinterpret_cast<const float4*>(fib)[nW];
        const int own = slab_of[x];
        int seen0 = -1, seen1 = -1;   // a slab is listed once (two slabs on a periodic axis are both neighbours)
#pragma unroll
        for (int ds_ = -1; ds_ <= 1; ++ds_) {
            int s = own + ds_;
            if (s < 0 || s >= n_slabs) {
                if (!(d.per & 1)) continue;
                s = (s + n_slabs) % n_slabs;
            }
            if (s == seen0 || s == seen1) continue;
            seen1 = seen0;
            seen0 = s;
            const int4 t = slab_tab[s];
            const int nxs = t.y - t.x + t.z + t.w;
            int lx = x - (t.x - t.z);
            if (d.per & 1) lx = ((lx % d.nx) + d.nx) % d.nx;
            if (lx < 0 || lx >= nxs) continue;
            const MemberDev& ds = mem[s];
            const long long n = ds.node_off + (lx + ds.px) + (long long)ds.NX * ((y + ds.py) + (long long)ds.NY * (z + ds.pz));
            reinterpret_cast<float4*>(fib)[n] = v;
            tag[n] = TAG_IB;
        }
    });
}

__global__ void __launch_bounds__(IB_MARKER_THREADS, IB_MARKER_MIN_BLOCKS)
k_ib_markers(const MemberDev* __restrict__ mem, uint8_t* __restrict__ tag, float* __restrict__ fib,
             const uint32_t* __restrict__ status, const int* __restrict__ v_cap, const CapsuleDev* __restrict__ caps,
             const CapsuleSums* __restrict__ sums, const float4* __restrict__ xm, const double* __restrict__ vel,
             const float* __restrict__ area, float* __restrict__ uv0, float* __restrict__ probe, int n_verts,
             const float4* __restrict__ macro) {
    // four lanes per marker
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = t & (GL - 1);
    const int l = min(t / GL, n_verts - 1);
    const int ax = min(r, 2);   // the axis this lane takes the nearest node of
    // the marker's coordinate (two-float mirror) and velocity along ax,
    // fetched beside its capsule's flags
    const float4 mh = xm[2 * l], ml = xm[2 * l + 1];
    const float Ph = ax == 0 ? mh.x : (ax == 1 ? mh.y : mh.z), Pl = ax == 0 ? ml.x : (ax == 1 ? ml.y : ml.z);
    const float Vb = (float)vel[3 * l + ax];
    const int cap = v_cap[l];
    const CapsuleDev& C = caps[cap];
    const int m = C.member;
    const bool valid = t / GL < n_verts && !(status[m] & STOP);
    const unsigned mask = __ballot_sync(FULL, valid);   // whole groups: validity is shared by a group
    if (!valid) return;
    const MemberDev& d = mem[m];
    MlsG M;
    float4 q[GS];
    mls_build_g<1, MARKER_FAST32>(d, macro, Ph, Pl, r, mask, M, q);
    float p[GS];
#pragma unroll
    for (int j = 0; j < GS; ++j) {
        const int k = r + GL * j;
        p[j] = k >= 27 ? 0.f : mls_row_g(M, 0, j, k);
    }
    float Ux = 0.f, Uy = 0.f, Uz = 0.f;
#pragma unroll
    for (int j = 0; j < GS; ++j) {
        Ux += p[j] * q[j].y; Uy += p[j] * q[j].z; Uz += p[j] * q[j].w;
    }
    Ux = group_sum(Ux, mask);
    Uy = group_sum(Uy, mask);
    Uz = group_sum(Uz, mask);
    const float Fx = __shfl_sync(mask, Vb, 0, GL) - Ux, Fy = __shfl_sync(mask, Vb, 1, GL) - Uy,
                Fz = __shfl_sync(mask, Vb, 2, GL) - Uz;
    const float A = area[l];
#pragma unroll
    for (int j = 0; j < GS; ++j) {
        if (p[j] != 0.f && q[j].x > 0.f) {
            // a fluid support node (the force a solid one would take acts on
            // the wall)
            const float c = A * p[j];
            const size_t gi = (size_t)d.node_off + mls_node_g(d, M, r + GL * j);
            // one vector reduction per support node (f_ib is padded to float4)
            atomicAdd(reinterpret_cast<float4*>(fib) + gi, make_float4(c * Fx, c * Fy, c * Fz, 0.f));
            // the shell pass flagged the fluid nodes of the capsule's band; a
            // block that leaves the box (its points clamped onto the box's
            // faces) or wraps a periodic seam flags its nodes itself
            if (M.base < 0) tag[gi] = TAG_IB;
        }
    }
    if (r == 0) {
        uv0[3 * l] = Ux; uv0[3 * l + 1] = Uy; uv0[3 * l + 2] = Uz;
        // volume penalty magnitude k_v (1 - V/V0) A, kept in the spare slot of
        // the + probe record; the update adds it along n
        float kvol = 0.f;
        if (!C.rigid) kvol = (float)(C.kv * (1.0 - sums[cap].V * C.inv_V0)) * A;
        probe[(size_t)2 * l * PROBE_STRIDE + 7] = kvol;
    }
}

__global__ void __launch_bounds__(IB_PROBE_THREADS, IB_PROBE_MIN_BLOCKS)
k_ib_probes(const MemberDev* __restrict__ mem, const uint8_t* __restrict__ tag, const uint32_t* __restrict__ status,
            const int* __restrict__ v_cap, const CapsuleDev* __restrict__ caps, const float4* __restrict__ xm,
            const float* __restrict__ nrm, float* __restrict__ probe, int n_verts,
            const float4* __restrict__ macro) {
    // four lanes per probe, two probes per marker: x + 1.2 n (s = 1), x - 1.2 n (s = 2)
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = t & (GL - 1);
    const int sid = t / GL;
    const int l = min(sid >> 1, n_verts - 1);
    const int s = 1 + (sid & 1);
    const int ax = min(r, 2);   // the axis this lane takes the nearest node of
    // the vertex coordinate (two-float mirror) and the normal along ax,
    // fetched beside its capsule's flags
    const float na = nrm[3 * l + ax];
    const float4 mh = xm[2 * l], ml = xm[2 * l + 1];
    const float xh = ax == 0 ? mh.x : (ax == 1 ? mh.y : mh.z), xl = ax == 0 ? ml.x : (ax == 1 ? ml.y : ml.z);
    const int m = caps[v_cap[l]].member;
    const bool valid = (sid >> 1) < n_verts && !(status[m] & STOP);
    const unsigned mask = __ballot_sync(FULL, valid);
    if (!valid) return;
    const MemberDev& d = mem[m];
    float ph, pl;
    probe_of(xh, xl, __fmul_rn(s == 1 ? 1.2f : -1.2f, na), ph, pl);
    MlsG M;
    float4 q[GS];
    mls_build_g<4, PROBE_FAST32>(d, macro, ph, pl, r, mask, M, q);
    float acc[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};   // rho, then grad u row-major
#pragma unroll
    for (int j = 0; j < GS; ++j) {
        const int k = r + GL * j;
        if (k >= 27) continue;
        const float p = mls_row_g(M, 0, j, k), g0 = mls_row_g(M, 1, j, k), g1 = mls_row_g(M, 2, j, k),
                    g2 = mls_row_g(M, 3, j, k);
        acc[0] += p * fabsf(q[j].x);   // a solid node's rho (1) is stored negated
        acc[1] += g0 * q[j].y; acc[2] += g1 * q[j].y; acc[3] += g2 * q[j].y;
        acc[4] += g0 * q[j].z; acc[5] += g1 * q[j].z; acc[6] += g2 * q[j].z;
        acc[7] += g0 * q[j].w; acc[8] += g1 * q[j].w; acc[9] += g2 * q[j].w;
    }
#pragma unroll
    for (int i = 0; i < 10; ++i) acc[i] = group_sum(acc[i], mask);
    if (r != 0) return;
    const float rP = acc[0];
    const float mu = rP * d.nu;
    float* rec = probe + ((size_t)2 * l + (s - 1)) * PROBE_STRIDE;
    rec[0] = rP * (1.f / 3.f);
    rec[1] = mu * 2.f * acc[1];
    rec[2] = mu * 2.f * acc[5];
    rec[3] = mu * 2.f * acc[9];
    rec[4] = mu * (acc[2] + acc[4]);
    rec[5] = mu * (acc[3] + acc[7]);
    rec[6] = mu * (acc[6] + acc[8]);
}


__global__ void __launch_bounds__(256) k_edges(const int* __restrict__ hinge, const int* __restrict__ e_cap,
                                               const CapsuleDev* __restrict__ caps, const uint32_t* __restrict__ status,
                                               const float4* __restrict__ xm, const float* __restrict__ l0,
                                               const float* __restrict__ ks, const float* __restrict__ th0,
                                               const float* __restrict__ kb, float* __restrict__ force, int n_edges) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n_edges) return;
    const CapsuleDev& C = caps[e_cap[e]];
    if (C.rigid || (status[C.member] & STOP)) return;
    const int4 hg = reinterpret_cast<const int4*>(hinge)[e];
    const int v1 = hg.x, v2 = hg.y, v3i = hg.z, v4 = hg.w;
    // positions relative to v2
    const f3 a = mirror_diff(xm, v1, v2), c = mirror_diff(xm, v3i, v2), dd = mirror_diff(xm, v4, v2);
    v3<float> F1, F2, F3, F4;
    hinge_forces<float>({a.x, a.y, a.z}, {c.x, c.y, c.z}, {dd.x, dd.y, dd.z}, ks[e], l0[e], kb[e], th0[e], F1, F2,
                        F3, F4);
    add_force(force, v1, {F1.x, F1.y, F1.z});
    add_force(force, v2, {F2.x, F2.y, F2.z});
    add_force(force, v3i, {F3.x, F3.y, F3.z});
    add_force(force, v4, {F4.x, F4.y, F4.z});
}

// ---------------------------------------------------------------------------
// Inter-body repulsion (Eq. collision) for markers of different capsules
// closer than 2 dx, found on a uniform grid of 2 dx cells.
//
// Broad phase first: a marker i of capsule c can be within 2 dx of a marker of
// capsule o only if it lies inside o's vertex box grown by 2 dx, and within
// R_o + 2 dx of o's reference point rc_o, R_o being the largest distance of
// o's vertices from rc_o (both from the geometry pass of this step).  k_broad
// lists, per capsule, the capsules of its lattice whose box grown by 3 meets
// its own box and whose sphere grown by 2 meets its own sphere; a marker
// outside the grown box or the grown sphere of every listed capsule neither
// enters the cell grid nor searches it.  The relation is symmetric, so every pair closer
// than the cutoff has both markers in the grid and both searching.  The boxes
// are those of the geometry pass at the same positions.  With the integer box
// [lo, hi] of o (lo <= x < hi for its vertices), a marker at X closer than 2
// to one of them has lo - 2 < X < hi + 2, hence lo - 2 <= floor(X) <= hi + 1;
// the test takes floor of X rounded to FP32 against [lo - 2, hi + 2], which
// holds whatever the rounding, in integer compares (GB300's FP64 pipe is
// narrow).
// ---------------------------------------------------------------------------
constexpr int NEAR_GROW = 3;   // capsule-level margin (cutoff 2 plus one node)
constexpr float NEAR_REACH = 2.01f;   // cutoff plus a slack for the FP32 distances

// R_o + NEAR_REACH, or infinity when a vertex was not finite
__device__ __forceinline__ float near_reach(const CapsuleSums& B) {
    const float r = sqrtf(__int_as_float(B.r2_hi)) + NEAR_REACH;
    return r < 1e6f ? r : INFINITY;
}

__global__ void __launch_bounds__(128) k_broad(const MemberDev* __restrict__ mem, const CapsuleDev* __restrict__ caps,
                                               const CapsuleSums* __restrict__ sums,
                                               const uint32_t* __restrict__ status, int4* __restrict__ near) {
    __shared__ int cnt;
    const int c = blockIdx.x;
    const int m = caps[c].member;
    const MemberDev& d = mem[m];
    int4* out = near + (size_t)c * NEAR_STRIDE;
    if (!d.has_cells || (status[m] & STOP)) {   // uniform over the block
        if (threadIdx.x == 0) out[0] = make_int4(0, 0, 0, 0);
        return;
    }
    if (threadIdx.x == 0) cnt = 0;
    __syncthreads();
    const CapsuleSums& A = sums[c];
    const float ra = near_reach(A);
    for (int o = d.cap_begin + threadIdx.x; o < d.cap_begin + d.cap_count; o += blockDim.x) {
        if (o == c) continue;
        const CapsuleSums& B = sums[o];
        bool meet = true;
#pragma unroll
        for (int a = 0; a < 3; ++a)
            meet = meet && A.box_lo[a] <= B.box_hi[a] + NEAR_GROW && B.box_lo[a] - NEAR_GROW <= A.box_hi[a];
        const float rb = near_reach(B);
        const float qx = A.rcf[0] - B.rcf[0], qy = A.rcf[1] - B.rcf[1], qz = A.rcf[2] - B.rcf[2];
        const float reach = ra + rb;   // R_A + R_B + 2 with slack (infinite if either is)
        meet = meet && qx * qx + qy * qy + qz * qz <= reach * reach;
        if (meet) {
            const int k = atomicAdd(&cnt, 1);
            if (k < NEAR_CAP) {
                out[1 + 3 * k] = make_int4(B.box_lo[0] - 2, B.box_lo[1] - 2, B.box_lo[2] - 2, 0);
                out[2 + 3 * k] = make_int4(B.box_hi[0] + 2, B.box_hi[1] + 2, B.box_hi[2] + 2, 0);
                out[3 + 3 * k] = make_int4(__float_as_int(B.rcf[0]), __float_as_int(B.rcf[1]), __float_as_int(B.rcf[2]),
                                           __float_as_int(rb));
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) out[0] = make_int4(cnt > NEAR_CAP ? -1 : cnt, 0, 0, 0);
}

// Whether a marker of capsule c at (X, Y, Z) lies inside the grown box and
// the grown sphere of a capsule listed as near c (always when the list
// overflowed).  The FP32 position is within 1e-3 of X below 1.6e4 lu, inside
// the sphere's 0.01 slack.
__device__ __forceinline__ bool near_other(const int4* __restrict__ near, int c, double X, double Y, double Z) {
    const int4* e = near + (size_t)c * NEAR_STRIDE;
    const int n = e[0].x;
    if (n < 0) return true;
    const float xf = (float)X, yf = (float)Y, zf = (float)Z;
    const int xi = (int)floorf(xf), yi = (int)floorf(yf), zi = (int)floorf(zf);
    for (int k = 0; k < n; ++k) {
        const int4 lo = e[1 + 3 * k], hi = e[2 + 3 * k], sp = e[3 + 3 * k];
        if (!(xi >= lo.x && xi <= hi.x && yi >= lo.y && yi <= hi.y && zi >= lo.z && zi <= hi.z)) continue;
        const float qx = xf - __int_as_float(sp.x), qy = yf - __int_as_float(sp.y), qz = zf - __int_as_float(sp.z);
        const float r = __int_as_float(sp.w);
        if (qx * qx + qy * qy + qz * qz <= r * r) return true;
    }
    return false;
}

__global__ void k_cells_fill(const MemberDev* __restrict__ mem, const int* __restrict__ v_cap, const CapsuleDev* __restrict__ caps,
                             const uint32_t* __restrict__ status, uint32_t* __restrict__ status_new,
                             const double* __restrict__ x, const int4* __restrict__ near, int* __restrict__ count,
                             float4* __restrict__ items, int* __restrict__ vids, int n_verts) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n_verts) return;
    const double X = x[3 * v], Y = x[3 * v + 1], Z = x[3 * v + 2];   // issued beside the capsule lookups
    const int cap = v_cap[v];
    const int m = caps[cap].member;
    const MemberDev& d = mem[m];
    if (!d.has_cells || (status[m] & STOP)) return;
    if (!near_other(near, cap, X, Y, Z)) return;
    const int cx = min(max((int)floor(X * 0.5), 0), d.cnx - 1);
    const int cy = min(max((int)floor(Y * 0.5), 0), d.cny - 1);
    const int cz = min(max((int)floor(Z * 0.5), 0), d.cnz - 1);
    const long long idx = d.cell_off + cx + (long long)d.cnx * (cy + (long long)d.cny * cz);
    const int slot = atomicAdd(count + idx, 1);
    // item: FP32 position (prefilter) and the capsule id; the vertex id beside it
    if (slot < CELL_CAP) {
        items[idx * CELL_CAP + slot] = make_float4((float)X, (float)Y, (float)Z, __int_as_float(cap));
        vids[idx * CELL_CAP + slot] = v;
    } else {
        atomicOr(status_new + m, ST_OVERFLOW);
    }
}

// RL lanes per marker: lane r searches cells k = r, r + RL, ... of the 27
// around the marker's cell, and the group sums the contributions.
constexpr int RL = 8;

__global__ void __launch_bounds__(256) k_repulsion(const MemberDev* __restrict__ mem, const int* __restrict__ v_cap,
                                                   const CapsuleDev* __restrict__ caps,
                                                   const uint32_t* __restrict__ status, const double* __restrict__ x,
                                                   const float* __restrict__ nrm, const int4* __restrict__ near,
                                                   const int* __restrict__ count, const float4* __restrict__ items,
                                                   const int* __restrict__ vids, float* __restrict__ force,
                                                   int n_verts) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = t / RL, r = t & (RL - 1);
    if (i >= n_verts) return;   // whole groups
    const double X = x[3 * i], Y = x[3 * i + 1], Z = x[3 * i + 2];   // issued beside the capsule lookups
    const int ci = v_cap[i];
    const int m = caps[ci].member;
    const MemberDev& d = mem[m];
    if (!d.has_cells || (status[m] & STOP)) return;
    if (!near_other(near, ci, X, Y, Z)) return;
    const unsigned gmask = ((1u << RL) - 1u) << ((threadIdx.x & 31) & ~(RL - 1));
    // the cell of the marker: lanes 0, 1, 2 take one axis each (FP64), the
    // group exchanges them
    const int ax = min(r, 2);
    const int cdim = ax == 0 ? d.cnx : (ax == 1 ? d.cny : d.cnz);
    const int ca = min(max((int)floor((ax == 0 ? X : (ax == 1 ? Y : Z)) * 0.5), 0), cdim - 1);
    const int cx = __shfl_sync(gmask, ca, 0, RL), cy = __shfl_sync(gmask, ca, 1, RL), cz = __shfl_sync(gmask, ca, 2, RL);
    const float Xf = (float)X, Yf = (float)Y, Zf = (float)Z;
    float acc = 0.f;
    for (int k = r; k < 27; k += RL) {
        const int qx = cx + sdx(k), qy = cy + sdy(k), qz = cz + sdz(k);
        if (qx < 0 || qy < 0 || qz < 0 || qx >= d.cnx || qy >= d.cny || qz >= d.cnz) continue;
        const long long idx = d.cell_off + qx + (long long)d.cnx * (qy + (long long)d.cny * qz);
        const int cnt = min(count[idx], CELL_CAP);
        for (int s = 0; s < cnt; ++s) {
            const float4 it = items[idx * CELL_CAP + s];
            if (__float_as_int(it.w) == ci) continue;   // same body
            // FP32 prefilter (coordinates below 1e4 lu round by < 1e-3, far
            // inside the 0.01 margin on d^2)
            const float fx = Xf - it.x, fy = Yf - it.y, fz = Zf - it.z;
            if (fx * fx + fy * fy + fz * fz > 4.01f) continue;
            const int j = vids[idx * CELL_CAP + s];
            // the cutoff decides a discontinuous force: take it in FP64
            const double rx = X - x[3 * j], ry = Y - x[3 * j + 1], rz = Z - x[3 * j + 2];
            const double d2 = rx * rx + ry * ry + rz * rz;
            if (d2 < 4.0) {
                const float dist = sqrtf((float)d2);
                acc += 1.f / (dist * dist * sqrtf(dist));
            }
        }
    }
#pragma unroll
    for (int o = 1; o < RL; o <<= 1) acc += __shfl_xor_sync(gmask, acc, o, RL);
    if (r == 0 && acc > 0.f) {
        const float c = d.umax * (1.f / (8.f * 1.41421356237f)) * acc;
        force[4 * i] -= c * nrm[3 * i];
        force[4 * i + 1] -= c * nrm[3 * i + 1];
        force[4 * i + 2] -= c * nrm[3 * i + 2];
    }
}

// ---------------------------------------------------------------------------
// Structure update.  Soft capsules, one thread per vertex: the Verlet
// predictor / velocity / corrector (Eqs. verletPos, verletVel, verletPosC) in
// FP64 on F^tot = hinge + repulsion + volume (accumulated in `force`) +
// hydrodynamic (probe records).  Rigid bodies, one block each: the
// Newton-Euler system with Eq. angularVelRig.  Then, one thread per edge, the
// damage rule (an edge at twice its rest length).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_verlet(const CapsuleDev* __restrict__ caps, const int* __restrict__ v_cap,
                                                const uint32_t* __restrict__ status, uint32_t* __restrict__ status_new,
                                                double* __restrict__ x, double* __restrict__ x_prev,
                                                double* __restrict__ vel, float* __restrict__ force,
                                                const float* __restrict__ uv0, const float* __restrict__ probe,
                                                const float* __restrict__ nrm, const float* __restrict__ area,
                                                float4* __restrict__ xm, int n_verts) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n_verts) return;
    const int cap = v_cap[v];
    // every per-vertex load is issued before the capsule's flags arrive, so
    // that their latencies overlap instead of following one another
    const float4 fo = reinterpret_cast<const float4*>(force)[v];
    double xt[3], xp[3];
    float u0[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        xt[a] = x[3 * v + a];
        xp[a] = x_prev[3 * v + a];
        u0[a] = uv0[3 * v + a];
    }
    float H[3];
    hydro_force(probe, nrm, area, v, H[0], H[1], H[2]);
    const CapsuleDev& C = caps[cap];
    if (C.rigid || (status[C.member] & STOP)) return;
    reinterpret_cast<float4*>(force)[v] = make_float4(0.f, 0.f, 0.f, 0.f);
    const float half_inv_m = 0.5f / (float)C.mv;
    const float F[3] = {fo.x, fo.y, fo.z};
    bool bad = false;
    double xn[3];
    // With a = F / (2 m_v): predictor x* = x + u_0 + a, velocity
    // u = 3/2 x* - 2 x + 1/2 x_prev = 3/2 (u_0 + a) + 1/2 (x_prev - x), corrector
    // x_new = x + u + a.  Positions stay FP64; the increments, of the size of
    // a velocity, are formed in FP32 (GB300's FP64 pipe is narrow).
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float acc = (F[a] + H[a]) * half_inv_m;
        const float back = (float)(xp[a] - xt[a]);
        const float un = 1.5f * (u0[a] + acc) + 0.5f * back;
        xn[a] = xt[a] + (double)(un + acc);
        x_prev[3 * v + a] = xt[a];
        x[3 * v + a] = xn[a];
        vel[3 * v + a] = (double)un;
        bad |= !isfinite(xn[a]);
    }
    mirror_put(xm, v, xn[0], xn[1], xn[2]);
    if (bad) atomicOr(status_new + C.member, ST_NONFINITE);
}

__global__ void __launch_bounds__(256) k_rigid(CapsuleDev* __restrict__ caps, const uint32_t* __restrict__ status,
                                               uint32_t* __restrict__ status_new, double* __restrict__ x,
                                               double* __restrict__ x_prev, double* __restrict__ vel,
                                               float* __restrict__ force, const float* __restrict__ probe,
                                               const float* __restrict__ nrm, const float* __restrict__ area,
                                               float4* __restrict__ xm) {
    __shared__ double red[32];
    __shared__ double sh_rig[16];
    CapsuleDev& C = caps[blockIdx.x];
    if (!C.rigid || (status[C.member] & STOP)) return;
    const int vb = C.v_begin, nv = C.v_count;
    const double xc0 = C.xc[0], xc1 = C.xc[1], xc2 = C.xc[2];
    double s[6] = {0, 0, 0, 0, 0, 0};
    for (int v = vb + threadIdx.x; v < vb + nv; v += blockDim.x) {
        float H[3];
        hydro_force(probe, nrm, area, v, H[0], H[1], H[2]);
        const double fx = (double)force[4 * v] + H[0], fy = (double)force[4 * v + 1] + H[1],
                     fz = (double)force[4 * v + 2] + H[2];
        force[4 * v] = 0.f; force[4 * v + 1] = 0.f; force[4 * v + 2] = 0.f;
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
    bool bad = false;
    for (int v = vb + threadIdx.x; v < vb + nv; v += blockDim.x) {
        const double rx = x[3 * v] - xc0, ry = x[3 * v + 1] - xc1, rz = x[3 * v + 2] - xc2;
        const double qx = R[0] * rx + R[1] * ry + R[2] * rz;
        const double qy = R[3] * rx + R[4] * ry + R[5] * rz;
        const double qz = R[6] * rx + R[7] * ry + R[8] * rz;
        x_prev[3 * v] = x[3 * v]; x_prev[3 * v + 1] = x[3 * v + 1]; x_prev[3 * v + 2] = x[3 * v + 2];
        x[3 * v] = ncx + qx; x[3 * v + 1] = ncy + qy; x[3 * v + 2] = ncz + qz;
        mirror_put(xm, v, ncx + qx, ncy + qy, ncz + qz);
        const double wx = sh_rig[12], wy = sh_rig[13], wz = sh_rig[14];
        vel[3 * v] = sh_rig[9] + (wy * qz - wz * qy);
        vel[3 * v + 1] = sh_rig[10] + (wz * qx - wx * qz);
        vel[3 * v + 2] = sh_rig[11] + (wx * qy - wy * qx);
        bad |= !(isfinite(x[3 * v]) && isfinite(x[3 * v + 1]) && isfinite(x[3 * v + 2]));
    }
    __syncthreads();
    if (threadIdx.x == 0) { C.xc[0] = ncx; C.xc[1] = ncy; C.xc[2] = ncz; }
    const int anybad = __syncthreads_or(bad ? 1 : 0);
    if (anybad && threadIdx.x == 0) atomicOr(status_new + C.member, ST_NONFINITE);
}

// l >= 2 l0 decided on squared lengths (no square root or division).
__global__ void __launch_bounds__(256) k_damage(const CapsuleDev* __restrict__ caps, const int* __restrict__ e_cap,
                                                const uint32_t* __restrict__ status, uint32_t* __restrict__ status_new,
                                                const float4* __restrict__ xm, const int* __restrict__ hinge,
                                                const float* __restrict__ l0, int n_edges) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n_edges) return;
    // the edge's vertices and positions are fetched before the capsule's
    // flags, so that the two chains of loads overlap
    const int4 h = reinterpret_cast<const int4*>(hinge)[e];
    const int a = h.y, b = h.z;
    const float l0e = l0[e];
    // the FP64 difference rounded to FP32 (two-float mirror), the squared
    // length in FP32 (a relative 1e-7 at the threshold of twice the rest length)
    const f3 r = mirror_diff(xm, a, b);
    const float dx = r.x, dy = r.y, dz = r.z;
    const CapsuleDev& C = caps[e_cap[e]];
    if (C.rigid || (status[C.member] & STOP)) return;
    if (dx * dx + dy * dy + dz * dz >= 4.f * l0e * l0e) atomicOr(status_new + C.member, ST_DAMAGED);
}

// ---------------------------------------------------------------------------
// FP64 diagnostics of every capsule (Section "Transport of an elastic
// capsule"; Reading R): per triangle, with a, b, c relative to the capsule's
// first vertex r0, v = a.(b x c)/6 and q = a + b + c: V += v, S += |N|/2,
// S1 += v q / 4, M2 += v/20 (a a^T + b b^T + c c^T + q q^T); per edge the
// largest l / l0; per vertex the summed velocity.  out holds per capsule
// V, S, S1[3], M2[6] (xx yy zz xy xz yz), vel[3], max stretch, r0[3].
// ---------------------------------------------------------------------------
constexpr int STAT_DOUBLES = CAP_STAT_DOUBLES;
constexpr int STAT_BLOCKS = 8;

__global__ void __launch_bounds__(256) k_capsule_stats(const CapsuleDev* __restrict__ caps, const double* __restrict__ x,
                                                       const double* __restrict__ vel, const int* __restrict__ tri,
                                                       const int* __restrict__ hinge, const float* __restrict__ l0,
                                                       int c_begin, double* __restrict__ out) {
    __shared__ double red[32];
    const int c = c_begin + blockIdx.x / STAT_BLOCKS, part = blockIdx.x % STAT_BLOCKS;
    const CapsuleDev& C = caps[c];
    const int r0 = C.v_begin;
    const double ox = x[3 * r0], oy = x[3 * r0 + 1], oz = x[3 * r0 + 2];
    double acc[STAT_DOUBLES];
    for (int i = 0; i < STAT_DOUBLES; ++i) acc[i] = 0.0;
    const int stride = STAT_BLOCKS * blockDim.x;
    for (int t = C.t_begin + part * blockDim.x + threadIdx.x; t < C.t_begin + C.t_count; t += stride) {
        const int ia = tri[3 * t], ib = tri[3 * t + 1], ic = tri[3 * t + 2];
        const double a[3] = {x[3 * ia] - ox, x[3 * ia + 1] - oy, x[3 * ia + 2] - oz};
        const double b[3] = {x[3 * ib] - ox, x[3 * ib + 1] - oy, x[3 * ib + 2] - oz};
        const double cc[3] = {x[3 * ic] - ox, x[3 * ic + 1] - oy, x[3 * ic + 2] - oz};
        const double bc[3] = {b[1] * cc[2] - b[2] * cc[1], b[2] * cc[0] - b[0] * cc[2], b[0] * cc[1] - b[1] * cc[0]};
        const double v = (a[0] * bc[0] + a[1] * bc[1] + a[2] * bc[2]) / 6.0;
        const double u[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]}, w[3] = {cc[0] - a[0], cc[1] - a[1], cc[2] - a[2]};
        const double N[3] = {u[1] * w[2] - u[2] * w[1], u[2] * w[0] - u[0] * w[2], u[0] * w[1] - u[1] * w[0]};
        const double q[3] = {a[0] + b[0] + cc[0], a[1] + b[1] + cc[1], a[2] + b[2] + cc[2]};
        acc[0] += v;
        acc[1] += 0.5 * sqrt(N[0] * N[0] + N[1] * N[1] + N[2] * N[2]);
        for (int k = 0; k < 3; ++k) acc[2 + k] += v * q[k] * 0.25;
        const int ii[6] = {0, 1, 2, 0, 0, 1}, jj[6] = {0, 1, 2, 1, 2, 2};
        for (int m = 0; m < 6; ++m)
            acc[5 + m] += v * 0.05 * (a[ii[m]] * a[jj[m]] + b[ii[m]] * b[jj[m]] + cc[ii[m]] * cc[jj[m]] +
                                      q[ii[m]] * q[jj[m]]);
    }
    for (int v = C.v_begin + part * blockDim.x + threadIdx.x; v < C.v_begin + C.v_count; v += stride)
        for (int k = 0; k < 3; ++k) acc[11 + k] += vel[3 * v + k];
    double mx = 0.0;
    for (int e = C.e_begin + part * blockDim.x + threadIdx.x; e < C.e_begin + C.e_count; e += stride) {
        const int4 h = reinterpret_cast<const int4*>(hinge)[e];
        const double dx = x[3 * h.y] - x[3 * h.z], dy = x[3 * h.y + 1] - x[3 * h.z + 1], dz = x[3 * h.y + 2] - x[3 * h.z + 2];
        mx = fmax(mx, sqrt(dx * dx + dy * dy + dz * dz) / (double)l0[e]);
    }
    double* o = out + (size_t)c * STAT_DOUBLES;
    for (int i = 0; i < 14; ++i) {
        const double t = block_sum_d(acc[i], red);
        if (threadIdx.x == 0) atomicAdd(o + i, t);
        __syncthreads();
    }
    // the largest stretch: non-negative doubles order as their bit patterns
#pragma unroll
    for (int off = 16; off; off >>= 1) mx = fmax(mx, __shfl_xor_sync(FULL, mx, off));
    if ((threadIdx.x & 31) == 0)
        atomicMax(reinterpret_cast<unsigned long long*>(o + 14), (unsigned long long)__double_as_longlong(mx));
    if (part == 0 && threadIdx.x == 0) { o[15] = ox; o[16] = oy; o[17] = oz; }
}

cudaError_t launch_capsule_stats(const DevState& d, int c_begin, int c_count, double* out, cudaStream_t s) {
    if (c_count <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(out + (size_t)c_begin * STAT_DOUBLES, 0, sizeof(double) * STAT_DOUBLES * c_count, s);
    if (e != cudaSuccess) return e;
    k_capsule_stats<<<c_count * STAT_BLOCKS, 256, 0, s>>>(d.caps, d.x, d.vel, d.tri, d.hinge, d.l0, c_begin, out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// launches
// ---------------------------------------------------------------------------
cudaError_t launch_geometry_snorm(const DevState& d, float* snorm, cudaStream_t s) {
    if (d.n_caps == 0) return cudaSuccess;
    k_geom_tri<<<d.n_caps * GEO_BLOCKS, 256, 0, s>>>(d.caps, d.sums, d.status, d.xm, d.tri, d.vacc);
    k_geom_vtx<<<(d.n_verts + 255) / 256, 256, 0, s>>>(d.caps, d.v_cap, d.sums, d.status, d.xm, d.vacc, d.nrm, d.area,
                                                       d.n_verts, snorm);
    return cudaGetLastError();
}

cudaError_t launch_geometry(const DevState& d, int, cudaStream_t s) { return launch_geometry_snorm(d, nullptr, s); }

template <typename T>
static cudaError_t shell_t(const DevState& d, int parity, cudaStream_t s) {
    bool lin = d.h_mem != nullptr;
    for (int m = 0; lin && m < d.n_members; ++m) lin = d.h_mem[m].per == 0 && !d.h_mem[m].slab_view;
    if (lin)
        k_shell<T, true><<<d.n_caps * SHELL_BLOCKS, 256, 0, s>>>(d.mem, (const T*)d.f, d.tag, d.status, d.caps,
                                                                 d.sums, d.macro, parity, d.fib, d.slab_of, d.slab_tab);
    else
        k_shell<T, false><<<d.n_caps * SHELL_BLOCKS, 256, 0, s>>>(d.mem, (const T*)d.f, d.tag, d.status, d.caps,
                                                                  d.sums, d.macro, parity, d.fib, d.slab_of, d.slab_tab);
    return cudaGetLastError();
}

cudaError_t launch_fib_scatter(const DevState& d, cudaStream_t s) {
    if (d.n_verts == 0 || d.slab_w < 0) return cudaSuccess;
    k_fib_scatter<<<d.n_caps * SHELL_BLOCKS, 256, 0, s>>>(d.mem, d.tag, d.fib, d.status, d.caps, d.sums, d.slab_of,
                                                          d.slab_tab, d.n_slabs);
    return cudaGetLastError();
}

cudaError_t launch_shell(const DevState& d, int parity, cudaStream_t s) {
    if (d.n_verts == 0) return cudaSuccess;
    switch (d.storage) {
        case 1: return shell_t<__half>(d, parity, s);
        case 2: return shell_t<__nv_bfloat16>(d, parity, s);
        default: return shell_t<float>(d, parity, s);
    }
}

cudaError_t launch_markers(const DevState& d, cudaStream_t s) {
    if (d.n_verts == 0) return cudaSuccess;
    const long long mt = (long long)GL * d.n_verts;
    k_ib_markers<<<(unsigned)((mt + IB_MARKER_THREADS - 1) / IB_MARKER_THREADS), IB_MARKER_THREADS, 0, s>>>(
        d.mem, d.tag, d.fib, d.status, d.v_cap, d.caps, d.sums, d.xm, d.vel, d.area, d.uv0, d.probe, d.n_verts,
        d.macro);
    return cudaGetLastError();
}

cudaError_t launch_probes(const DevState& d, cudaStream_t s) {
    if (d.n_verts == 0) return cudaSuccess;
    const long long pt = 2LL * GL * d.n_verts;
    k_ib_probes<<<(unsigned)((pt + IB_PROBE_THREADS - 1) / IB_PROBE_THREADS), IB_PROBE_THREADS, 0, s>>>(
        d.mem, d.tag, d.status, d.v_cap, d.caps, d.xm, d.nrm, d.probe, d.n_verts, d.macro);
    return cudaGetLastError();
}

cudaError_t launch_edges(const DevState& d, cudaStream_t s) {
    if (!d.any_soft || d.n_edges == 0) return cudaSuccess;
    k_edges<<<(d.n_edges + 255) / 256, 256, 0, s>>>(d.hinge, d.e_cap, d.caps, d.status, d.xm, d.l0, d.ks, d.th0, d.kb,
                                                     d.force, d.n_edges);
    return cudaGetLastError();
}

cudaError_t launch_repulsion(const DevState& d, cudaStream_t s) {
    if (!d.any_cells) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(d.cell_count, 0, sizeof(int) * d.n_cells, s);
    if (e != cudaSuccess) return e;
    const int blocks = (d.n_verts + 255) / 256;
    k_broad<<<d.n_caps, 128, 0, s>>>(d.mem, d.caps, d.sums, d.status, d.near);
    k_cells_fill<<<blocks, 256, 0, s>>>(d.mem, d.v_cap, d.caps, d.status, d.status_new, d.x, d.near, d.cell_count,
                                        d.cell_items, d.cell_vid, d.n_verts);
    const long long rt = (long long)RL * d.n_verts;
    k_repulsion<<<(unsigned)((rt + 255) / 256), 256, 0, s>>>(d.mem, d.v_cap, d.caps, d.status, d.x, d.nrm, d.near,
                                                             d.cell_count, d.cell_items, d.cell_vid, d.force,
                                                             d.n_verts);
    return cudaGetLastError();
}

cudaError_t launch_update(const DevState& d, cudaStream_t s) {
    if (d.n_caps == 0) return cudaSuccess;
    if (d.any_soft)
        k_verlet<<<(d.n_verts + 255) / 256, 256, 0, s>>>(d.caps, d.v_cap, d.status, d.status_new, d.x, d.x_prev, d.vel,
                                                         d.force, d.uv0, d.probe, d.nrm, d.area, d.xm, d.n_verts);
    if (d.any_rigid)
        k_rigid<<<d.n_caps, 256, 0, s>>>(d.caps, d.status, d.status_new, d.x, d.x_prev, d.vel, d.force, d.probe, d.nrm,
                                         d.area, d.xm);
    if (d.any_soft && d.n_edges > 0)
        k_damage<<<(d.n_edges + 255) / 256, 256, 0, s>>>(d.caps, d.e_cap, d.status, d.status_new, d.xm, d.hinge, d.l0,
                                                         d.n_edges);
    return cudaGetLastError();
}

cudaError_t launch_mirror(const DevState& d, cudaStream_t s) {
    if (d.n_verts == 0) return cudaSuccess;
    k_mirror<<<(d.n_verts + 255) / 256, 256, 0, s>>>(d.x, d.xm, d.n_verts);
    return cudaGetLastError();
}

}  // namespace ibl
