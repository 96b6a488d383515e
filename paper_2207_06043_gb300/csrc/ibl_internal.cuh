// Internal device/host definitions of libibl (not part of the C ABI).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <string>

namespace ibl {

// ---------------------------------------------------------------------------
// D3Q19 velocity set of Eq. e_i, packed two bits per direction so that both
// compile-time (unrolled) and run-time (per-link) lookups are pure ALU work.
// component(k) = ((CODE >> 2k) & 3) - 1
// ---------------------------------------------------------------------------
constexpr uint64_t EX_CODE = 0x15402a9549ull;
constexpr uint64_t EY_CODE = 0x294949495ull;
constexpr uint64_t EZ_CODE = 0x889494955ull;

__host__ __device__ constexpr int ex(int k) { return int((EX_CODE >> (2 * k)) & 3ull) - 1; }
__host__ __device__ constexpr int ey(int k) { return int((EY_CODE >> (2 * k)) & 3ull) - 1; }
__host__ __device__ constexpr int ez(int k) { return int((EZ_CODE >> (2 * k)) & 3ull) - 1; }
// opposite direction: pairs (1,2) (3,4) (5,6) (7,12) (8,11) (9,14) (10,13) (15,18) (16,17)
__host__ __device__ constexpr int opp(int k) {
    return k == 0 ? 0
         : k <= 6 ? ((k & 1) ? k + 1 : k - 1)
         : (k == 7 || k == 8 || k == 11 || k == 12) ? 19 - k
         : k <= 14 ? 23 - k
         : 33 - k;
}
__host__ __device__ constexpr float wgt(int k) {
    return k == 0 ? (1.0f / 3.0f) : (k <= 6 ? (1.0f / 18.0f) : (1.0f / 36.0f));
}

constexpr int Q = 19;
constexpr uint32_t LINK_AT_FACE = 128u;   // l_meta flag: the link starts on a Zou-He face node
constexpr int MAX_MEMBERS = 128;

enum : uint8_t { TAG_SOLID = 1, TAG_IB = 2 };
enum : uint32_t { ST_DAMAGED = 1, ST_NONFINITE = 2, ST_OVERFLOW = 4,
                  ST_TIMEOUT = 8 };   // a bounded device wait gave up
enum { FACE_NONE = 0, FACE_VELOCITY = 1, FACE_PRESSURE = 2,
       FACE_HALO = 3 };   // a cut face of a slab member: its planes are copied from their owner

// Per-lattice descriptor (a device array per context, passed to every kernel).
struct MemberDev {
    int nx, ny, nz;          // user dims
    int NX, NY, NZ;          // padded dims (non-periodic axes get a ghost layer)
    int px, py, pz;          // padding per axis (0 periodic, 1 otherwise)
    int per;                 // bit a set: axis a periodic
    int N;                   // padded node count
    int S;                   // plane stride in elements
    long long f_off;         // element offset of plane 0 of this member
    long long node_off;      // offset into per-node arrays (tag, f_ib)
    float omega, guo, nu, umax;
    float F[3];
    int hasF;                // nonzero body force
    float st_scale, ld_scale;
    int face_kind[6];
    float face_rho[6];
    long long face_off[6];   // float3 record offset into the face velocity array
    int seg_begin, seg_count;    // range of this member in the interior-segment list
    int bseg_begin, bseg_count;  // and in the border-segment list
    int link_begin, link_count;
    int cap_begin, cap_count;
    int vert_begin, vert_count;
    long long cell_off;
    int cnx, cny, cnz, has_cells;
    int slab_view;           // 1: the whole lattice of a slab context, seen by its capsules (no populations)
};

// Per-capsule descriptor (global memory).
struct CapsuleDev {
    int member;
    int rigid;
    int v_begin, v_count;
    int t_begin, t_count;
    int e_begin, e_count;
    double kv, V0, inv_V0, S0, mass, mv, inertia;
    double xc[3], u1[3], u2[3], w1[3], w2[3];
};

// Per-capsule FP64 sums written each step / on demand.
struct CapsuleSums {
    double V, S;
    double cen[3];           // sum v (a+b+c)/4 relative to ref
    double M2[6];            // xx yy zz xy xz yz relative to ref
    double ref[3];
    double max_stretch;
    int box_lo[3], box_hi[3];   // integer bounding box of the vertices (user coordinates)
    double rc[3];               // reference point of the step: centre of the previous step's box
    float rcf[3];               // the same in FP32 (a half-integer: exact)
    int r2_lo, r2_hi;           // FP32 bits of the least / largest squared vertex distance from rc
};

// ---------------------------------------------------------------------------
// storage conversion
// ---------------------------------------------------------------------------
template <typename T> struct Store;
template <> struct Store<float> {
    static __device__ __forceinline__ float ld(const float* p, float) { return *p; }
    static __device__ __forceinline__ void st(float* p, float v, float) { *p = v; }
};
template <> struct Store<__half> {
    static __device__ __forceinline__ float ld(const __half* p, float s) { return __half2float(*p) * s; }
    static __device__ __forceinline__ void st(__half* p, float v, float s) { *p = __float2half_rn(v * s); }
};
template <> struct Store<__nv_bfloat16> {
    static __device__ __forceinline__ float ld(const __nv_bfloat16* p, float) { return __bfloat162float(*p); }
    static __device__ __forceinline__ void st(__nv_bfloat16* p, float v, float) { *p = __float2bfloat16_rn(v); }
};

// ---------------------------------------------------------------------------
// host-side launch entry points (one per translation unit)
// ---------------------------------------------------------------------------
// Device buffers of a context (all members concatenated).
constexpr uint32_t NO_NODE = 0xffffffffu;   // padding entry of the lattice work lists

struct DevState {
    int storage = 0;                 // 0 f32, 1 f16, 2 bf16
    int n_members = 0;
    const MemberDev* h_mem = nullptr;
    MemberDev* mem = nullptr;         // device copy of the member table (one per context)
    int threads = 128;               // lattice kernel threads per block (one warp per group of 32 nodes)
    // 32-node segments holding at least one fluid node, all members, split
    // into interior ones and border ones (a fluid node on a periodic wrap
    // plane); entries are segment indices (padded node / 32) within their
    // member.  The adjoint sweep runs over these.
    int n_segs = 0, n_bsegs = 0;
    uint32_t* segs = nullptr;
    uint32_t* bsegs = nullptr;
    // Work lists of the lattice kernel: the fluid nodes of each member
    // (padded index within the member) in ascending order, interior ones and
    // wrap-plane ones apart, each member's list padded with NO_NODE to a
    // multiple of 32; one warp per group of 32 entries.
    int n_groups = 0, n_bgroups = 0;
    uint32_t* nodes = nullptr;
    uint32_t* bnodes = nullptr;
    int* group_mem = nullptr;        // member of each group (batched contexts; null with one member)
    int* bgroup_mem = nullptr;
    int lbm_blocks = 0, lbm_bblocks = 0;   // ceil(groups / (threads / 32))
    // staged lattice kernel (single-lattice contexts): the interior fluid
    // nodes as chunks (first node, nodes) of consecutive nodes, at most
    // lbm_chunk_nodes() each; resident blocks per SM of that kernel (0: not
    // available)
    int n_chunks = 0;
    uint2* chunks = nullptr;
    int bulk_blocks_per_sm = 0;
    int lattice_path = 0;            // 1: staged kernel where available, 0: register gathers
    int grid_lbm = 0;                // persistent grid of the interior kernel (0: default)
    int n_sm = 0;                    // multiprocessors of the device

    void* f = nullptr;               // 19 planes per member, f - w
    size_t f_bytes = 0;
    uint8_t* tag = nullptr;          // per padded node
    float* fib = nullptr;            // float4 (x, y, z, pad) per padded node, zero outside the IB shell
    float* face_vel = nullptr;       // float3 per face node of velocity faces
    uint32_t* status = nullptr;      // per member, constant during a step
    uint32_t* status_new = nullptr;  // flags raised during a step, merged at the next step begin
    int* counters = nullptr;         // steps completed, per member

    int n_face_nodes = 0;            // fluid nodes on a Zou-He face, all members
    uint32_t* fc_node = nullptr;     // padded node
    uint32_t* fc_meta = nullptr;     // face | member << 8
    int* fc_lbeg = nullptr;          // n_face_nodes + 1: the face node's wall links in fc_links
    int* fc_links = nullptr;         // link indices (their l_meta carries LINK_AT_FACE)

    int n_links = 0;
    uint32_t* l_node = nullptr;      // padded node of the link
    uint32_t* l_meta = nullptr;      // dir | ok1 << 5 | ok2 << 6 | LINK_AT_FACE | member << 8
    float* l_q = nullptr;
    float* l_dq = nullptr;           // dq / d(junction radius) per link (adjoint input)

    int n_caps = 0, n_verts = 0, n_tris = 0, n_edges = 0;
    int any_soft = 0, any_rigid = 0, any_cells = 0, max_nv = 0;
    CapsuleDev* caps = nullptr;
    CapsuleSums* sums = nullptr;
    int* v_cap = nullptr;
    double* x = nullptr;             // 3 per vertex
    double* x_prev = nullptr;
    double* vel = nullptr;
    float* force = nullptr;          // float4 per vertex (x, y, z, pad): hinge + repulsion forces, cleared by the update
    float* uv0 = nullptr;            // 3 per vertex
    float* nrm = nullptr;            // 3 per vertex
    float* area = nullptr;           // per vertex
    float4* macro = nullptr;         // (rho, u*) per padded node, written in capsule shells
    float* probe = nullptr;          // 2 probe records (8 floats) per vertex
    float4* vacc = nullptr;          // per-vertex normal / area accumulator, zero between steps
    int* tri = nullptr;              // 3 per triangle (global vertex ids)
    int* hinge = nullptr;            // 4 per edge: v1 v2 v3 v4 (edge = v2-v3)
    float* l0 = nullptr;
    float* ks = nullptr;
    float* th0 = nullptr;
    float* kb = nullptr;
    int* e_cap = nullptr;
    int* cell_count = nullptr;
    float4* cell_items = nullptr;    // (x, y, z, capsule id bits) per slot
    int* cell_vid = nullptr;         // vertex id per slot
    float4* xm = nullptr;            // two-float mirror of x: (hi, 0), (lo, 0) per vertex, x = hi + lo
    int4* near = nullptr;            // NEAR_STRIDE per capsule: count (-1: too many), then grown boxes and spheres
    long long n_cells = 0;
    // slab decomposition: plane copies (dst member, dst padded x, src member,
    // src padded x) run after every step; members share NY and NZ
    int n_halo = 0;
    int4* halo = nullptr;
    // capsules of a slab context live in the whole-lattice member slab_w:
    // its moments are taken from the slab owning each node (slab_of, per
    // global x) and its IB force is copied to every slab holding the node
    int slab_w = -1, n_slabs = 0;
    const int* slab_of = nullptr;
    const int4* slab_tab = nullptr;     // (x0, x1, lo, hi) per slab
};
constexpr int CELL_CAP = 32;
constexpr int NEAR_CAP = 31;          // capsules listed as near one capsule; more: all its markers search
constexpr int NEAR_STRIDE = 1 + 3 * NEAR_CAP;   // int4 entries: the count, then three per listed capsule


// The optional tape pointers record, per step, what the discrete adjoint needs
// from the forward state: (rho, u) of every fluid node before the collision
// (float4 per padded node), d(value)/dq of every wall link, rho of every face
// node before the face rule.  Null in ordinary steps.
cudaError_t launch_lbm(const DevState& d, int parity, cudaStream_t s, float4* tape_rhou = nullptr,
                       float4* tape_F = nullptr);
int lbm_max_threads();   // block-size bound the lattice kernel was compiled for
// the staged lattice kernel (lbm_bulk.cu): whether the context's layout
// allows it, its set-up (shared-memory attribute; resident blocks per SM) and
// its launch over the interior groups of a single lattice
bool lbm_bulk_layout_ok(const DevState& d);
cudaError_t lbm_bulk_prepare(int storage, int& blocks_per_sm);
int lbm_chunk_nodes();
cudaError_t launch_lbm_bulk(const DevState& d, int parity, cudaStream_t s);
// the wall fill (Eq. bbouzidi) and the Zou-He faces (Eq. extbound) of the
// step just done, in one launch
cudaError_t launch_walls(const DevState& d, int parity_done, cudaStream_t s, float* tape_dvdq = nullptr,
                         float* tape_rho = nullptr);
cudaError_t launch_init_member(const DevState& d, int m, const float* rho, const float* u, cudaStream_t s);
cudaError_t launch_read(const DevState& d, int member, int parity, float* rho, float* u,
                        float* g, cudaStream_t s);

// discrete adjoint of the lattice step (adjoint.cu)
cudaError_t launch_adj_objective(const DevState& d, int parity, const int lo[3], const int hi[3], const double w[3],
                                 float* lam, size_t LS, double* J, cudaStream_t s);
cudaError_t launch_adj_step(const DevState& d, const float* tape_rho, const float* tape_dvdq, const float4* tape_rhou,
                            float* lam_in, float* lam_out, size_t LS, double* grad_s, double* grad_q,
                            cudaStream_t s, const float4* tape_F = nullptr, float4* lam_fib = nullptr);

cudaError_t launch_geometry(const DevState& d, int full, cudaStream_t s);
// the same, also recording |S_l| (the length of each vertex's unnormalised
// normal) when snorm is not null
cudaError_t launch_geometry_snorm(const DevState& d, float* snorm, cudaStream_t s);

// Capsule adjoint (adjoint_ib.cu): per-vertex adjoint vectors, the per-node
// lambda_F of the lattice adjoint and the support-node accumulators.
struct AdjCapPtrs {
    float4 *lx = nullptr, *lxp = nullptr, *lv = nullptr, *lU = nullptr, *lF = nullptr, *ln = nullptr;
    float *lA = nullptr, *snorm = nullptr;
    double* lV = nullptr;
    float4 *lfib = nullptr, *lmac = nullptr;
    double* acc_ca = nullptr;
};
// geometry of x(t) (already in the vertex arrays) for a reverse step, with the
// volume adjoint reset
cudaError_t launch_adj_geometry(const DevState& d, double* lV, float* snorm, cudaStream_t s);
// the capsule part of a reverse step t (after the lattice part wrote lam and
// p.lfib), with the lattice tape of step t and the vertex velocities at t
cudaError_t launch_adj_capsules(const DevState& d, const AdjCapPtrs& p, const float4* tape_rhou, const float4* tape_F,
                                const double* vel_t, float* lam, size_t LS, cudaStream_t s);
// IB pass: shell moments, then the marker stencils (interpolation, force,
// spreading) and the probe stencils (stresses), which are independent of
// each other (the markers set only the IB bit of fluid tags, the probes read
// only the solid bit; they write different slots of the probe records).
cudaError_t launch_shell(const DevState& d, int parity, cudaStream_t s);
cudaError_t launch_markers(const DevState& d, cudaStream_t s);
cudaError_t launch_probes(const DevState& d, cudaStream_t s);
cudaError_t launch_step_begin(const DevState& d, cudaStream_t s);
cudaError_t launch_edges(const DevState& d, cudaStream_t s);
cudaError_t launch_repulsion(const DevState& d, cudaStream_t s);
cudaError_t launch_update(const DevState& d, cudaStream_t s);
// refresh the two-float mirror of the vertex positions after x is set from the host
cudaError_t launch_mirror(const DevState& d, cudaStream_t s);
// FP64 sums of capsules c_begin .. c_begin + c_count - 1 into out (18 doubles
// per capsule: V, S, S1[3] and M2[6] about the first vertex r0, summed
// velocity[3], max stretch, r0[3])
constexpr int CAP_STAT_DOUBLES = 18;
cudaError_t launch_capsule_stats(const DevState& d, int c_begin, int c_count, double* out, cudaStream_t s);
// the halo planes of a slab decomposition from their owners (every slot of
// every padded node of each listed plane)
cudaError_t launch_halo(const DevState& d, cudaStream_t s);
// the IB force spread into the whole-lattice member of a slab context, to the
// slabs that hold each node (owner and ghost copies), before the lattice step
cudaError_t launch_fib_scatter(const DevState& d, cudaStream_t s);
// the stop flags raised on those capsules, to every slab
cudaError_t launch_status_spread(const DevState& d, cudaStream_t s);

// marker-based wall tagging and BFL distances (walls.cu): 0, or -1 (argument)
// / -3 (CUDA) with msg set; arguments as ibl_voxelise_markers
int voxelise_markers(const double* verts, int nv, const int32_t* tris, int nt, int nx, int ny, int nz,
                     const int32_t* periodic, const uint8_t* tag_in, uint8_t* tag_out, uint32_t* link_node,
                     uint32_t* link_dir, float* link_q, int64_t* n_links, cudaStream_t s, std::string& msg);

}  // namespace ibl
