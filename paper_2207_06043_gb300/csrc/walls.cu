// Tagging of a lattice by a triangulated fixed wall and the BFL distances
// measured to the wall's markers (Section "Boundary conditions on fixed
// bodies", Eq. qbouzidi).  A set-up pass: it produces the cell tags and the
// wall links that ibl_set_geometry takes, so the quadratic bounce-back of the
// step runs unchanged on them.
//
// The rule: the markers are the triangle centroids; a node whose cell holds a
// marker is solid; a node that is not solid and sees a solid node at x + e_i
// gets a wall link in direction i with q = |x_b - x_L| / |e_i|, x_L the marker
// of the solid cell nearest to x_b.  A solid node that holds no marker (solid
// beforehand, e.g. a box edge) gives q = 1/2; q is clipped to [1e-6, 1].
// The cell of a node is the unit cube centred on it (a marker at c lies in the
// cell of floor(c + 1/2) per axis).  Every integer decision and every
// distance is taken in FP64 with explicitly rounded operations (no
// contraction), and q is rounded to FP32 once.
#include <cstdint>
#include <string>
#include <vector>

#include "ibl_internal.cuh"

namespace ibl {
namespace {

struct Box {
    int n[3];
    int per[3];
};

__device__ __forceinline__ bool wrap(long long& c, int n, int per) {
    if (per) {
        c %= n;
        if (c < 0) c += n;
        return true;
    }
    return c >= 0 && c < n;
}

__device__ __forceinline__ void centroid(const double* __restrict__ V, const int* __restrict__ T, int t,
                                         double L[3]) {
    const int a = T[3 * t], b = T[3 * t + 1], c = T[3 * t + 2];
#pragma unroll
    for (int ax = 0; ax < 3; ++ax)
        L[ax] = __ddiv_rn(__dadd_rn(__dadd_rn(V[3 * a + ax], V[3 * b + ax]), V[3 * c + ax]), 3.0);
}

// the raw (unwrapped) node of the marker's cell, and its flat index if the
// cell lies in the box (or wraps onto it); -1 otherwise
__device__ __forceinline__ long long marker_cell(const double L[3], const Box& B, long long raw[3]) {
    long long c[3];
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        raw[ax] = (long long)floor(__dadd_rn(L[ax], 0.5));
        c[ax] = raw[ax];
        if (!wrap(c[ax], B.n[ax], B.per[ax])) return -1;
    }
    return c[0] + (long long)B.n[0] * (c[1] + (long long)B.n[1] * c[2]);
}

__global__ void k_vox_mark(const double* __restrict__ V, const int* __restrict__ T, int nt, Box B,
                           uint8_t* __restrict__ tag) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nt; t += gridDim.x * blockDim.x) {
        double L[3];
        long long raw[3];
        centroid(V, T, t, L);
        const long long s = marker_cell(L, B, raw);
        if (s >= 0) tag[s] = TAG_SOLID;
    }
}

// per node: the 18-bit mask of directions i (bit i-1) whose neighbour is solid,
// for nodes that are not solid themselves, and its population count
__global__ void k_vox_mask(const uint8_t* __restrict__ tag, Box B, long long N, uint32_t* __restrict__ mask,
                           uint32_t* __restrict__ cnt) {
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N;
         n += (long long)gridDim.x * blockDim.x) {
        uint32_t m = 0;
        if (tag[n] == 0) {
            const long long x = n % B.n[0], y = (n / B.n[0]) % B.n[1], z = n / ((long long)B.n[0] * B.n[1]);
            for (int i = 1; i < Q; ++i) {
                long long c[3] = {x + ex(i), y + ey(i), z + ez(i)};
                bool in = true;
#pragma unroll
                for (int ax = 0; ax < 3; ++ax) in = in && wrap(c[ax], B.n[ax], B.per[ax]);
                if (in && tag[c[0] + (long long)B.n[0] * (c[1] + (long long)B.n[1] * c[2])] != 0) m |= 1u << (i - 1);
            }
        }
        mask[n] = m;
        cnt[n] = __popc(m);
    }
}

// exclusive scan of cnt within blocks of 1024 (one element per thread); the
// block totals go to tot
__global__ void __launch_bounds__(1024) k_vox_scan(uint32_t* __restrict__ cnt, long long N,
                                                   uint32_t* __restrict__ tot) {
    __shared__ uint32_t warp_sum[32];
    const long long n = blockIdx.x * 1024ll + threadIdx.x;
    const uint32_t v = n < N ? cnt[n] : 0u;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t s = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t u = __shfl_up_sync(0xffffffffu, s, o);
        if (lane >= o) s += u;
    }
    if (lane == 31) warp_sum[w] = s;
    __syncthreads();
    if (w == 0) {
        uint32_t t = warp_sum[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t u = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += u;
        }
        warp_sum[lane] = t;
    }
    __syncthreads();
    const uint32_t before = (w ? warp_sum[w - 1] : 0u) + s - v;
    if (n < N) cnt[n] = before;
    if (threadIdx.x == 1023) tot[blockIdx.x] = warp_sum[31];
}

__global__ void k_vox_scan_add(uint32_t* __restrict__ base, long long N, const uint32_t* __restrict__ off) {
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N;
         n += (long long)gridDim.x * blockDim.x)
        base[n] += off[n >> 10];
}

__global__ void k_vox_links(const uint32_t* __restrict__ mask, const uint32_t* __restrict__ base, long long N,
                            uint32_t* __restrict__ lnode, uint32_t* __restrict__ ldir,
                            unsigned long long* __restrict__ dist) {
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N;
         n += (long long)gridDim.x * blockDim.x) {
        uint32_t m = mask[n];
        uint32_t j = base[n];
        while (m) {
            const int b = __ffs(m) - 1;
            m &= m - 1;
            lnode[j] = (uint32_t)n;
            ldir[j] = (uint32_t)(b + 1);
            dist[j] = 0x7ff0000000000000ull;      // +inf: no marker seen yet
            ++j;
        }
    }
}

// every marker offers |x_b - x_L| to each boundary node b = x_s - e_i of its
// cell; a link keeps the smallest (non-negative doubles order as their bits)
__global__ void k_vox_q(const double* __restrict__ V, const int* __restrict__ T, int nt, Box B,
                        const uint8_t* __restrict__ tag, const uint32_t* __restrict__ mask,
                        const uint32_t* __restrict__ base, unsigned long long* __restrict__ dist) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nt; t += gridDim.x * blockDim.x) {
        double L[3];
        long long raw[3];
        centroid(V, T, t, L);
        if (marker_cell(L, B, raw) < 0) continue;
        for (int i = 1; i < Q; ++i) {
            const long long br[3] = {raw[0] - ex(i), raw[1] - ey(i), raw[2] - ez(i)};
            long long c[3] = {br[0], br[1], br[2]};
            bool in = true;
#pragma unroll
            for (int ax = 0; ax < 3; ++ax) in = in && wrap(c[ax], B.n[ax], B.per[ax]);
            if (!in) continue;
            const long long b = c[0] + (long long)B.n[0] * (c[1] + (long long)B.n[1] * c[2]);
            if (tag[b] != 0) continue;
            const uint32_t m = mask[b];
            const uint32_t bit = 1u << (i - 1);
            if (!(m & bit)) continue;
            const uint32_t j = base[b] + __popc(m & (bit - 1u));
            const double dx = __dadd_rn((double)br[0], -L[0]);
            const double dy = __dadd_rn((double)br[1], -L[1]);
            const double dz = __dadd_rn((double)br[2], -L[2]);
            const double d = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz)));
            atomicMin(dist + j, (unsigned long long)__double_as_longlong(d));
        }
    }
}

__global__ void k_vox_finish(const uint32_t* __restrict__ ldir, const unsigned long long* __restrict__ dist,
                             long long nl, float* __restrict__ q) {
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < nl;
         j += (long long)gridDim.x * blockDim.x) {
        const int i = (int)ldir[j];
        const double d = __longlong_as_double((long long)dist[j]);
        const double elen = (i <= 6) ? 1.0 : 1.4142135623730951;   // |e_i|, sqrt(2) rounded to nearest
        double v = isinf(d) ? 0.5 : __ddiv_rn(d, elen);
        v = fmin(fmax(v, 1e-6), 1.0);
        q[j] = __double2float_rn(v);
    }
}

template <typename T>
struct DevBuf {
    T* p = nullptr;
    ~DevBuf() {
        if (p) cudaFree(p);
    }
    cudaError_t alloc(size_t n) { return cudaMalloc((void**)&p, sizeof(T) * (n ? n : 1)); }
};

int grid_for(long long n, int threads) {
    const long long b = (n + threads - 1) / threads;
    return (int)(b < 1 ? 1 : (b > 152ll * 64 ? 152ll * 64 : b));
}

}  // namespace

// returns 0 on success, -1 (argument), -3 (CUDA) with msg set
int voxelise_markers(const double* verts, int nv, const int32_t* tris, int nt, int nx, int ny, int nz,
                     const int32_t* periodic, const uint8_t* tag_in, uint8_t* tag_out, uint32_t* link_node,
                     uint32_t* link_dir, float* link_q, int64_t* n_links, cudaStream_t s, std::string& msg) {
    if (!n_links || !tag_out || nx < 1 || ny < 1 || nz < 1 || nv < 0 || nt < 0 || (nt > 0 && (!verts || !tris))) {
        msg = "ibl_voxelise_markers: bad arguments";
        return -1;
    }
    const long long N = (long long)nx * ny * nz;
    if (N >= (1ll << 32) / 19) {
        msg = "ibl_voxelise_markers: box too large for 32-bit link indices";
        return -1;
    }
    for (long long k = 0; k < 3ll * nt; ++k)
        if (tris[k] < 0 || tris[k] >= nv) {
            msg = "ibl_voxelise_markers: triangle index out of range";
            return -1;
        }
    Box B{{nx, ny, nz}, {periodic && periodic[0] ? 1 : 0, periodic && periodic[1] ? 1 : 0,
                         periodic && periodic[2] ? 1 : 0}};
#define VCK(call)                                                              \
    do {                                                                       \
        cudaError_t e_ = (call);                                               \
        if (e_ != cudaSuccess) {                                               \
            msg = std::string(#call) + ": " + cudaGetErrorString(e_);          \
            return -3;                                                         \
        }                                                                      \
    } while (0)
    DevBuf<double> dV;
    DevBuf<int> dT;
    DevBuf<uint8_t> dtag;
    DevBuf<uint32_t> dmask, dbase, dtot;
    VCK(dV.alloc(3ull * nv));
    VCK(dT.alloc(3ull * nt));
    VCK(dtag.alloc(N));
    VCK(dmask.alloc(N));
    VCK(dbase.alloc(N));
    const long long nblk = (N + 1023) / 1024;
    VCK(dtot.alloc(nblk));
    if (nv) VCK(cudaMemcpyAsync(dV.p, verts, sizeof(double) * 3 * nv, cudaMemcpyHostToDevice, s));
    if (nt) VCK(cudaMemcpyAsync(dT.p, tris, sizeof(int) * 3 * nt, cudaMemcpyHostToDevice, s));
    if (tag_in) VCK(cudaMemcpyAsync(dtag.p, tag_in, N, cudaMemcpyHostToDevice, s));
    else VCK(cudaMemsetAsync(dtag.p, 0, N, s));
    if (nt) k_vox_mark<<<grid_for(nt, 256), 256, 0, s>>>(dV.p, dT.p, nt, B, dtag.p);
    k_vox_mask<<<grid_for(N, 256), 256, 0, s>>>(dtag.p, B, N, dmask.p, dbase.p);
    k_vox_scan<<<(unsigned)nblk, 1024, 0, s>>>(dbase.p, N, dtot.p);
    VCK(cudaGetLastError());
    std::vector<uint32_t> tot(nblk), off(nblk);
    VCK(cudaMemcpyAsync(tot.data(), dtot.p, sizeof(uint32_t) * nblk, cudaMemcpyDeviceToHost, s));
    VCK(cudaStreamSynchronize(s));
    unsigned long long acc = 0;
    for (long long b = 0; b < nblk; ++b) {
        off[b] = (uint32_t)acc;
        acc += tot[b];
    }
    const long long nl = (long long)acc;
    const bool want = link_node || link_dir || link_q;
    if (want && (!link_node || !link_dir || !link_q || *n_links < nl)) {
        *n_links = nl;
        msg = "ibl_voxelise_markers: link buffers missing or smaller than the link count";
        return -1;
    }
    *n_links = nl;
    VCK(cudaMemcpyAsync(tag_out, dtag.p, N, cudaMemcpyDeviceToHost, s));
    if (!want || nl == 0) {
        VCK(cudaStreamSynchronize(s));
        return 0;
    }
    VCK(cudaMemcpyAsync(dtot.p, off.data(), sizeof(uint32_t) * nblk, cudaMemcpyHostToDevice, s));
    k_vox_scan_add<<<grid_for(N, 256), 256, 0, s>>>(dbase.p, N, dtot.p);
    DevBuf<uint32_t> dnode, ddir;
    DevBuf<unsigned long long> ddist;
    DevBuf<float> dq;
    VCK(dnode.alloc(nl));
    VCK(ddir.alloc(nl));
    VCK(ddist.alloc(nl));
    VCK(dq.alloc(nl));
    k_vox_links<<<grid_for(N, 256), 256, 0, s>>>(dmask.p, dbase.p, N, dnode.p, ddir.p, ddist.p);
    if (nt) k_vox_q<<<grid_for(nt, 256), 256, 0, s>>>(dV.p, dT.p, nt, B, dtag.p, dmask.p, dbase.p, ddist.p);
    k_vox_finish<<<grid_for(nl, 256), 256, 0, s>>>(ddir.p, ddist.p, nl, dq.p);
    VCK(cudaGetLastError());
    VCK(cudaMemcpyAsync(link_node, dnode.p, sizeof(uint32_t) * nl, cudaMemcpyDeviceToHost, s));
    VCK(cudaMemcpyAsync(link_dir, ddir.p, sizeof(uint32_t) * nl, cudaMemcpyDeviceToHost, s));
    VCK(cudaMemcpyAsync(link_q, dq.p, sizeof(float) * nl, cudaMemcpyDeviceToHost, s));
    VCK(cudaStreamSynchronize(s));
#undef VCK
    return 0;
}

}  // namespace ibl
