// Halo exchange of a slab decomposition along x (ibl_slab_group_create):
// one copy kernel, after every step, for the ghost planes of all slabs.
#include <algorithm>
#include <cstdint>

#include "ibl_internal.cuh"

namespace ibl {

// ---------------------------------------------------------------------------
// Halo planes of a slab decomposition along x.  Every step ends with each
// member's ghost planes overwritten by the planes of the members that own
// them: all 19 slots of every padded node of the plane (fluid and solid, so
// that the wall values the bounce-back left in solid slots travel too).  The
// pair index runs fastest, so that the consecutive ghost planes of one side
// (consecutive in memory) go to consecutive lanes.
// ---------------------------------------------------------------------------
template <typename E>
__global__ void k_halo(const MemberDev* __restrict__ mem, E* __restrict__ f, const int4* __restrict__ halo, int n_pairs,
                       int NY, long long n_plane) {
    const long long total = (long long)n_pairs * n_plane * Q;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int p = (int)(t % n_pairs);
        const long long r = t / n_pairs;
        const long long yz = r % n_plane;
        const int k = (int)(r / n_plane);
        const int4 h = halo[p];
        const MemberDev& dd = mem[h.x];
        const MemberDev& ds = mem[h.z];
        const long long Y = yz % NY, Z = yz / NY;
        const long long nd = h.y + (long long)dd.NX * (Y + (long long)NY * Z);
        const long long ns = h.w + (long long)ds.NX * (Y + (long long)NY * Z);
        f[dd.f_off + (long long)k * dd.S + nd] = f[ds.f_off + (long long)k * ds.S + ns];
    }
}

cudaError_t launch_halo(const DevState& d, cudaStream_t s) {
    if (d.n_halo == 0) return cudaSuccess;
    const MemberDev& m0 = d.h_mem[0];
    const long long n_plane = (long long)m0.NY * m0.NZ;
    const long long total = (long long)d.n_halo * n_plane * Q;
    const int threads = 256;
    const long long want = (total + threads - 1) / threads;
    const int blocks = (int)std::min<long long>(want, (long long)std::max(d.n_sm, 1) * 16);
    if (d.storage == 0)
        k_halo<uint32_t><<<blocks, threads, 0, s>>>(d.mem, (uint32_t*)d.f, d.halo, d.n_halo, m0.NY, n_plane);
    else
        k_halo<uint16_t><<<blocks, threads, 0, s>>>(d.mem, (uint16_t*)d.f, d.halo, d.n_halo, m0.NY, n_plane);
    return cudaGetLastError();
}

// The flags a step raised on the capsules of a slab context (their member is
// the whole-lattice view) stop every slab at the next step begin.
__global__ void k_status_spread(uint32_t* __restrict__ status_new, int n_members, int w) {
    const int m = threadIdx.x;
    if (m < n_members && m != w) {
        const uint32_t f = status_new[w];
        if (f) atomicOr(status_new + m, f);
    }
}

cudaError_t launch_status_spread(const DevState& d, cudaStream_t s) {
    if (d.slab_w < 0) return cudaSuccess;
    k_status_spread<<<1, MAX_MEMBERS, 0, s>>>(d.status_new, d.n_members, d.slab_w);
    return cudaGetLastError();
}

}  // namespace ibl
