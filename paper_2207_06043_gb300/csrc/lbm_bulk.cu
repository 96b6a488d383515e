// Lattice step (Eq. evoleq, collide + AA-pattern stream) with the gathers
// staged in shared memory by bulk copies.
//
// The register-gather kernel (lbm.cu) keeps 19 loads per lane in flight, so
// its bytes in flight per SM are bounded by its registers and occupancy.
// Here the interior fluid nodes of a single lattice are cut into chunks: runs
// of consecutive nodes of at most CH = 32 * TILE_WARPS nodes (every run of the
// work list is split into such pieces).  A chunk needs, for every population,
// one contiguous span of slots (the AA parity decides the plane and the
// offset) and one span of tag bytes, so a block fetches it with Q + 1 bulk
// copies of the spans' 16-byte-aligned supersets into one of TILE_STAGES
// shared-memory buffers.  One producer warp per block issues the copies
// (one lane per span) several chunks ahead; TILE_WARPS consumer warps take
// one node per lane from the buffer, collide and store from registers as
// the register kernel does.  A full barrier per buffer completes when its
// copies have landed, an empty barrier when every consumer warp has read it.
//
// Waits on the barriers are bounded in time: a wait that runs out raises
// ST_TIMEOUT for the lattice, waits (bounded again) for the copies still in
// flight into the warp's buffers and ends the warp; the host then reports
// IBL_ERR_TIMEOUT.
#include <cstdint>

#include "lbm_device.cuh"

#ifndef TILE_WARPS
#define TILE_WARPS 4          // consumer warps per block (a chunk is 32 * TILE_WARPS nodes at most)
#endif
#ifndef TILE_STAGES
#define TILE_STAGES 4         // buffers per block (chunks in flight)
#endif
#ifndef TILE_ALIGN
#define TILE_ALIGN 16         // alignment (bytes) of every copied superset and buffer row
#endif
#ifndef TILE_MIN_BLOCKS
#define TILE_MIN_BLOCKS 5     // resident blocks per SM the kernel is compiled for
#endif

namespace ibl {

namespace {

// a bounded wait gives up after this many SM clock cycles (about 1 s)
constexpr long long WAIT_CYCLES = 2000000000LL;

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_barrier_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(b)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_to_smem(void* dst, const void* src, uint32_t bytes, uint64_t* b) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(b))
        : "memory");
}
// shared-memory loads by address (the shared path, not a generic load)
__device__ __forceinline__ uint32_t lds_b32(uint32_t a) {
    uint32_t v;
    asm volatile("ld.shared.b32 %0, [%1];" : "=r"(v) : "r"(a) : "memory");
    return v;
}
__device__ __forceinline__ uint32_t lds_b16(uint32_t a) {
    unsigned short v;
    asm volatile("ld.shared.b16 %0, [%1];" : "=h"(v) : "r"(a) : "memory");
    return v;
}
__device__ __forceinline__ uint32_t lds_u8(uint32_t a) {
    uint32_t v;
    asm volatile("ld.shared.u8 %0, [%1];" : "=r"(v) : "r"(a) : "memory");
    return v;
}
__device__ __forceinline__ uint2 lds_v2(uint32_t a) {
    uint2 v;
    asm volatile("ld.shared.v2.b32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "r"(a) : "memory");
    return v;
}
__device__ __forceinline__ void sts_v2(uint32_t a, uint2 v) {
    asm volatile("st.shared.v2.b32 [%0], {%1, %2};" ::"r"(a), "r"(v.x), "r"(v.y) : "memory");
}
// a stored population from its bits (the storage scaling of Store<T>)
template <typename T> struct SmemPop;
template <> struct SmemPop<float> {
    static __device__ __forceinline__ float ld(uint32_t a, float) { return __uint_as_float(lds_b32(a)); }
};
template <> struct SmemPop<__half> {
    static __device__ __forceinline__ float ld(uint32_t a, float s) {
        return __half2float(__ushort_as_half((unsigned short)lds_b16(a))) * s;
    }
};
template <> struct SmemPop<__nv_bfloat16> {
    static __device__ __forceinline__ float ld(uint32_t a, float) {
        return __bfloat162float(__ushort_as_bfloat16((unsigned short)lds_b16(a)));
    }
};

__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(b)) : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t* b, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(b)), "r"(parity)
        : "memory");
    return ok != 0;
}
// every lane waits for the phase of the given parity; false (for the whole
// warp) when a lane ran out of time
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* b, uint32_t parity) {
    bool ok = mbar_test(b, parity);
    if (!ok) {
        const long long t0 = clock64();
        while (!(ok = mbar_test(b, parity)))
            if (clock64() - t0 > WAIT_CYCLES) break;
    }
    return __all_sync(0xffffffffu, ok);
}

template <typename T>
struct TileShape {
    static constexpr int A = TILE_ALIGN;
    static constexpr int CH = 32 * TILE_WARPS;            // nodes of a chunk at most
    // a span and its alignment slack, whole aligned units
    static constexpr int ROW_BYTES = (CH * (int)sizeof(T) + 2 * A + A - 1) / A * A;
    static constexpr int TAG_BYTES = (CH + 2 * A + A - 1) / A * A;
    static constexpr int STAGE_BYTES = Q * ROW_BYTES + TAG_BYTES;
    static constexpr int BAR_OFF = TILE_STAGES * STAGE_BYTES;
    static constexpr int DESC_OFF = BAR_OFF + 2 * TILE_STAGES * 8;   // (first node, nodes) of each buffer's chunk
    static constexpr int BLOCK_BYTES = DESC_OFF + TILE_STAGES * 8;
    static_assert(A % 16 == 0 && ROW_BYTES % 16 == 0 && STAGE_BYTES % 16 == 0, "16-byte rows");
};

// element index of the first slot of population k's span for a run starting
// at node n0 (parity 0: slot k of the nodes themselves; parity 1: slot
// opp(k) of the upstream nodes n - e_k)
__device__ __forceinline__ long long span_index(const MemberDev& d, int n0, int k, int parity) {
    return parity == 0 ? (long long)k * d.S + n0 : (long long)opp(k) * d.S + (n0 - lin_off(d, k));
}

// the producer warp: the bulk copies of a chunk (len nodes from n0) into
// stage buffer buf, completing on barrier bar; lane k < Q copies population
// k's span, lane Q the tags' span, lane 0 first posts the expected bytes
template <typename T>
__device__ __forceinline__ void issue_chunk(const MemberDev& d, const T* __restrict__ fm,
                                            const uint8_t* __restrict__ tag, int n0, int len, int parity,
                                            unsigned char* buf, uint64_t* bar, int lane) {
    using B = TileShape<T>;
    uintptr_t a = 0, src = 0;
    uint32_t bytes = 0;
    unsigned char* dst = buf + Q * B::ROW_BYTES;
    if (lane < Q) {
        a = reinterpret_cast<uintptr_t>(fm + span_index(d, n0, lane, parity));
        bytes = (uint32_t)len * (uint32_t)sizeof(T);
        dst = buf + lane * B::ROW_BYTES;
    } else if (lane == Q) {
        a = reinterpret_cast<uintptr_t>(tag + n0);
        bytes = (uint32_t)len;
    }
    if (bytes) {
        src = a & ~(uintptr_t)(B::A - 1);
        bytes = (uint32_t)(((a + bytes + B::A - 1) & ~(uintptr_t)(B::A - 1)) - src);
    }
    const uint32_t total = __reduce_add_sync(0xffffffffu, bytes);
    if (lane == 0) mbar_expect_tx(bar, total);
    __syncwarp();
    if (bytes) bulk_to_smem(dst, reinterpret_cast<const void*>(src), bytes, bar);
}

}  // namespace

// One time step of the interior fluid nodes of a single lattice (the
// wrap-plane nodes take the register kernel's border launch).  chunk[c] =
// (first node, nodes) of chunk c; block b takes chunks b, b + gridDim.x, ...
template <typename T>
__global__ void __launch_bounds__((TILE_WARPS + 1) * 32, TILE_MIN_BLOCKS)
k_lbm_tile(const __grid_constant__ MemberDev d, T* __restrict__ f, uint8_t* __restrict__ tag,
           float* __restrict__ fib, const uint32_t* __restrict__ status, uint32_t* __restrict__ status_new,
           const uint2* __restrict__ chunk, int n_chunks, int parity) {
    using B = TileShape<T>;
    extern __shared__ __align__(1024) unsigned char smem[];
    if (status[0] & (ST_DAMAGED | ST_NONFINITE)) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + B::BAR_OFF);
    uint64_t* empty = full + TILE_STAGES;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int s = 0; s < TILE_STAGES; ++s) {
            mbar_init(full + s, 1);
            mbar_init(empty + s, TILE_WARPS);
        }
        fence_barrier_init();
    }
    __syncthreads();
    const T* fm = f;
    bool failed = false;
    int j = 0;
    const uint32_t desc_s = smem_addr(smem + B::DESC_OFF);
    if (warp == TILE_WARPS) {
        // producer: refill buffer j % STAGES once every consumer warp has
        // read the chunk it held.  The chunk descriptors come 32 iterations
        // at a time (lane l holds iteration jb + l), the next batch loaded a
        // batch ahead; each one is handed to the consumers in shared memory
        // before the buffer's copies are posted
        auto batch = [&](int jb) -> uint2 {
            const int c = blockIdx.x + (jb + lane) * gridDim.x;
            return c < n_chunks ? __ldg(chunk + c) : make_uint2(0u, 0u);
        };
        uint2 cur = batch(0), nxt = batch(32);
        for (;; ++j) {
            if (j > 0 && (j & 31) == 0) {
                cur = nxt;
                nxt = batch(j + 32);
            }
            const int c = blockIdx.x + j * gridDim.x;
            if (c >= n_chunks) break;
            const int s = j % TILE_STAGES;
            const uint2 ch = make_uint2(__shfl_sync(0xffffffffu, cur.x, j & 31), __shfl_sync(0xffffffffu, cur.y, j & 31));
            if (j >= TILE_STAGES && !mbar_wait_bounded(empty + s, ((j / TILE_STAGES) - 1) & 1)) {
                failed = true;
                break;
            }
            if (lane == 0) sts_v2(desc_s + 8 * s, ch);
            issue_chunk<T>(d, fm, tag, (int)ch.x, (int)ch.y, parity, smem + s * B::STAGE_BYTES, full + s, lane);
        }
        // a producer that gave up leaves the consumers' waits to run out
        if (failed && lane == 0) atomicOr(status_new, ST_TIMEOUT);
        return;
    }
    for (;; ++j) {
        const int c = blockIdx.x + j * gridDim.x;
        if (c >= n_chunks) break;
        const int s = j % TILE_STAGES;
        if (!mbar_wait_bounded(full + s, (j / TILE_STAGES) & 1)) { failed = true; break; }
        const uint2 ch = lds_v2(desc_s + 8 * s);
        const uint32_t buf = smem_addr(smem + s * B::STAGE_BYTES);
        const int i = 32 * warp + lane;
        const bool act = i < (int)ch.y;
        const int n0 = (int)ch.x, n = n0 + i;
        float gv[Q];
        uint8_t tg = 0;
        if (act) {
#pragma unroll
            for (int k = 0; k < Q; ++k) {
                const uintptr_t a = reinterpret_cast<uintptr_t>(fm + span_index(d, n0, k, parity));
                const uint32_t sh = (uint32_t)(a & (B::A - 1));   // bytes before the span in its row
                gv[k] = SmemPop<T>::ld(buf + k * B::ROW_BYTES + sh + (uint32_t)i * sizeof(T), d.ld_scale);
            }
            tg = (uint8_t)lds_u8(buf + Q * B::ROW_BYTES + (uint32_t)(reinterpret_cast<uintptr_t>(tag + n0) & (B::A - 1)) + i);
        }
        // this warp is done with the buffer
        __syncwarp();
        if (lane == 0) mbar_arrive(empty + s);
        if (!act) continue;
        const bool ibn = tg & TAG_IB;
        float Fx = d.F[0], Fy = d.F[1], Fz = d.F[2];
        bool hasF = d.hasF != 0;
        if (ibn) {
            const float4 fv = reinterpret_cast<const float4*>(fib)[n];
            Fx += fv.x; Fy += fv.y; Fz += fv.z;
            reinterpret_cast<float4*>(fib)[n] = make_float4(0.f, 0.f, 0.f, 0.f);
            tag[n] = tg & (uint8_t)~TAG_IB;
            hasF = true;
        }
        collide(gv, d.omega, d.guo, Fx, Fy, Fz, hasF);
        store_post_lin<T>(d, f, n, parity, gv);
    }
    if (failed) {
        if (lane == 0) atomicOr(status_new, ST_TIMEOUT);
        // let the copies the producer may have issued into the next buffers
        // land before the block's shared memory is released
        for (int jj = j; jj < j + TILE_STAGES; ++jj)
            if (blockIdx.x + jj * gridDim.x < n_chunks) mbar_wait_bounded(full + jj % TILE_STAGES, (jj / TILE_STAGES) & 1);
    }
}

namespace {

template <typename T>
cudaError_t lbm_bulk_t(const DevState& d, int parity, cudaStream_t s) {
    using B = TileShape<T>;
    static_assert(B::BLOCK_BYTES <= 227 * 1024, "stage buffers exceed the shared memory of a block");
    if (d.n_chunks == 0) return cudaSuccess;
    const int grid = std::min(d.n_chunks, d.bulk_blocks_per_sm * d.n_sm);
    k_lbm_tile<T><<<grid, (TILE_WARPS + 1) * 32, B::BLOCK_BYTES, s>>>(d.h_mem[0], (T*)d.f, d.tag, d.fib, d.status,
                                                                      d.status_new, d.chunks, d.n_chunks, parity);
    return cudaGetLastError();
}

template <typename T>
cudaError_t bulk_prepare_t(int& blocks_per_sm) {
    using B = TileShape<T>;
    cudaError_t e = cudaFuncSetAttribute(k_lbm_tile<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, B::BLOCK_BYTES);
    if (e != cudaSuccess) return e;
    int nb = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_lbm_tile<T>, (TILE_WARPS + 1) * 32, B::BLOCK_BYTES);
    if (e != cudaSuccess) return e;
    blocks_per_sm = nb;
    return cudaSuccess;
}

}  // namespace

int lbm_chunk_nodes() { return 32 * TILE_WARPS; }

bool lbm_bulk_layout_ok(const DevState& d) {
    // every span's 16-byte superset must start inside the populations and the
    // planes must keep the 16-byte alignment of the buffer
    const size_t es = d.storage == 0 ? 4 : 2;
    if (d.n_members != 1 || !d.h_mem) return false;
    const MemberDev& m = d.h_mem[0];
    return m.f_off == 0 && ((size_t)m.S * es) % 16 == 0 && (reinterpret_cast<uintptr_t>(d.f) & 15u) == 0 &&
           (reinterpret_cast<uintptr_t>(d.tag) & 15u) == 0;
}

cudaError_t lbm_bulk_prepare(int storage, int& blocks_per_sm) {
    switch (storage) {
        case 1: return bulk_prepare_t<__half>(blocks_per_sm);
        case 2: return bulk_prepare_t<__nv_bfloat16>(blocks_per_sm);
        default: return bulk_prepare_t<float>(blocks_per_sm);
    }
}

cudaError_t launch_lbm_bulk(const DevState& d, int parity, cudaStream_t s) {
    switch (d.storage) {
        case 1: return lbm_bulk_t<__half>(d, parity, s);
        case 2: return lbm_bulk_t<__nv_bfloat16>(d, parity, s);
        default: return lbm_bulk_t<float>(d, parity, s);
    }
}

}  // namespace ibl
