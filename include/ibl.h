/*
 * ibl.h - C ABI of the GB300 lattice-Boltzmann / dynamic-immersed-boundary
 * solver (Coclite, de Tullio, Pascazio, Politi, "Characterization of
 * micro-Capsules Deformation in Branching Channels").
 *
 * One call of ibl_step advances every lattice of a context by whole time steps
 * of the coupled method:
 *   - D3Q19 BGK collide + stream (Eq. evoleq, Eq. eqfunc) with the Guo forcing
 *     term of the immersed-boundary force (Eq. forcing);
 *   - Zou-He velocity / pressure conditions on the box faces (Eq. extbound);
 *   - quadratic Bouzidi-Firdaouss-Lallemand bounce-back on fixed walls
 *     (Eq. qbouzidi, Eq. bbouzidi);
 *   - moving-least-squares interpolation / spreading between capsule mesh
 *     vertices and the lattice (Eqs. uLag, l2norm, intKernel, bodyforce);
 *   - spring-network membrane, volume penalty, probe-based hydrodynamic
 *     stresses and inter-body repulsion (Eqs. strainPot .. collision);
 *   - Verlet update of soft capsules (Eqs. verletPos .. verletPosC) and the
 *     Newton-Euler update of rigid bodies (Eq. angularVelRig);
 *   - the damage rule of Section "Transport of an elastic capsule": a mesh edge
 *     at twice its rest length stops the run.
 *
 * Conventions
 *   - Lattice units: dx = dt = 1, reference density 1, p = rho/3.
 *   - Node index = x + nx*(y + ny*z) (x fastest).
 *   - Direction numbering is the one of Eq. e_i.
 *   - Faces: 0 = x-, 1 = x+, 2 = y-, 3 = y+, 4 = z-, 5 = z+.  A face array is
 *     laid out with the lower remaining axis fastest (face 0/1: y + ny*z,
 *     face 2/3: x + nx*z, face 4/5: x + nx*y).
 *   - Ownership: the library copies every input; outputs go to caller
 *     buffers.  A buffer flagged on_device is a device pointer that the
 *     library reads/writes on the context's stream.
 *   - Errors: every call returns an ibl_status; ibl_last_error gives the text.
 *     No call throws across the ABI.  CUDA failures return IBL_ERR_CUDA.
 *   - The library owns all device memory of a context (allocated with
 *     cudaMalloc when the context is first stepped or read) and frees it in
 *     ibl_destroy.
 */
#ifndef IBL_H
#define IBL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ibl_ctx ibl_ctx;

typedef enum {
    IBL_OK = 0,
    IBL_ERR_ARG = -1,        /* invalid argument or inconsistent geometry      */
    IBL_ERR_OOM = -2,        /* device or host allocation failed               */
    IBL_ERR_CUDA = -3,       /* a CUDA runtime call failed                      */
    IBL_ERR_DAMAGED = -4,    /* a capsule edge reached twice its rest length   */
    IBL_ERR_NONFINITE = -5,  /* a vertex position became NaN/Inf               */
    IBL_ERR_TIMEOUT = -6,    /* a bounded device wait gave up (staged step)    */
    IBL_ERR_STATE = -7       /* call not allowed in the context's current state */
} ibl_status;

/* storage of the distributions f_i - w_i (arithmetic is always FP32) */
enum { IBL_STORAGE_F32 = 0, IBL_STORAGE_F16 = 1, IBL_STORAGE_BF16 = 2 };
/* Dirichlet kind of a box face (Section "Dirichlet conditions ...") */
enum { IBL_FACE_NONE = 0, IBL_FACE_VELOCITY = 1, IBL_FACE_PRESSURE = 2 };

typedef struct {
    int32_t nx, ny, nz;      /* lattice nodes per axis (each >= 3)               */
    int32_t storage;         /* IBL_STORAGE_*                                    */
    int32_t periodic[3];     /* nonzero: the axis wraps                          */
    int32_t reserved;
    double tau;              /* BGK relaxation time; nu = (tau - 1/2)/3 (> 0.5)  */
    double body_force[3];    /* uniform force density added to f_ib              */
    double u_max;            /* characteristic velocity of Eq. collision         */
} ibl_lattice_desc;

/* A fixed-wall link (Eq. qbouzidi): node + e_dir is solid and the wall cuts the
 * link at fraction q in (0, 1] of its length, measured from node.  dq is the
 * derivative of q with respect to the geometry parameter (kept for the
 * gradient path; ignored by the forward step). */
typedef struct {
    uint32_t node;
    uint32_t dir;
    float q;
    float dq;
} ibl_wall_link;

/* Capsule material (Section "Deforming bodies constitutive model"):
 * k_s0 = rho nu u_ref / Ca, k_s,l = k_s0 (A_a + A_b) / l0^2,
 * k_b = Eb k_s,l r^2 (r = radius of the rest volume), volume penalty kv,
 * mass = density_ratio * rest volume.  rigid != 0: Newton-Euler body. */
typedef struct {
    double Ca, Eb, kv, density_ratio, u_ref;
    int32_t rigid;
    int32_t reserved;
} ibl_capsule_params;

/* FP64 capsule diagnostics at the current state. */
typedef struct {
    double centroid[3];      /* volume centroid                                   */
    double volume, area;     /* enclosed volume, surface area                      */
    double dS;               /* (S - S0)/S0, the relative stretching of Section 2 */
    double taylor_D;         /* (a_max - a_min)/(a_max + a_min), equivalent ellipsoid */
    double max_stretch;      /* max edge length / rest length                      */
    double semi_axes[3];     /* ascending                                          */
    double velocity[3];      /* mean vertex velocity                               */
    int32_t damaged;
    int32_t reserved;
} ibl_capsule_stats;

/* Create a context with one lattice.  cuda_stream: a cudaStream_t (NULL = the
 * legacy default stream); every device operation of the context runs on it.
 * The context belongs to the CUDA device current at this call; that device
 * must be current at every later call (IBL_ERR_STATE when the context is set
 * up on another).  Until the first ibl_step / ibl_read_* the context holds
 * host data only. */
ibl_status ibl_create(const ibl_lattice_desc* desc, void* cuda_stream, ibl_ctx** out);

/* Fixed geometry (Section "No-Slip boundary conditions for stationary immersed
 * boundaries"): cell_tag[nx*ny*nz] 0 = fluid, 1 = solid; links as above (only
 * fluid nodes whose neighbour along dir is solid and inside the box).  Every
 * fluid node on a non-periodic face must lie on exactly one face. */
ibl_status ibl_set_geometry(ibl_ctx* ctx, const uint8_t* cell_tag,
                            const ibl_wall_link* links, size_t n_links);

/* Velocity face: u_xyz[3 * n_face] (face layout, x,y,z per node) is imposed
 * on the fluid nodes of the face (Eq. extbound). */
ibl_status ibl_set_inlet_velocity(ibl_ctx* ctx, int32_t face, const float* u_xyz);

/* Pressure face: density rho_out with zero tangential velocity. */
ibl_status ibl_set_outlet_pressure(ibl_ctx* ctx, int32_t face, double rho_out);

/* Initial populations at equilibrium with rho[N] and u[3N] (x,y,z per node);
 * either may be NULL (rho = 1, u = 0).  Default: rest state. */
ibl_status ibl_init_equilibrium(ibl_ctx* ctx, const float* rho, const float* u);

/* Add a closed triangular mesh (verts[3*nv] FP64, tris[3*nt] outward CCW)
 * whose vertices are the Lagrangian markers.  vel0[3] may be NULL.
 * IBL_ERR_ARG here for a vertex index out of range or repeated within a
 * triangle; a mesh that is not closed or not consistently oriented is
 * reported (IBL_ERR_ARG, naming the capsule) when the context is set up. */
ibl_status ibl_add_capsule(ibl_ctx* ctx, const double* verts, int32_t nv,
                           const int32_t* tris, int32_t nt, const double* vel0,
                           const ibl_capsule_params* params, int32_t* id_out);

/* Advance n_steps time steps.  steps_done (may be NULL) receives the steps
 * member 0 completed.  Returns IBL_ERR_DAMAGED when a capsule broke (the state
 * stays readable and the damaged lattice stops stepping), IBL_ERR_NONFINITE
 * when a vertex left the finite range, IBL_ERR_TIMEOUT when a wait of the
 * staged lattice kernel gave up (see ibl_set_lattice_path). */
ibl_status ibl_step(ibl_ctx* ctx, int32_t n_steps, int32_t* steps_done);

/* Macroscopic fields of member 0: rho[N], u[3N] (either may be NULL), with
 * rho u = sum f e + F_body/2; solid nodes read 0.  Host buffers that are
 * page-locked (cudaHostAlloc / cudaMallocHost, or a pinned torch tensor) are
 * written by the read kernel directly.  Other host buffers take the values
 * through a device staging buffer that the context allocates on the first
 * such read (cudaMalloc), keeps, and grows when a later read needs more;
 * ibl_destroy frees it. */
ibl_status ibl_read_fields(ibl_ctx* ctx, float* rho, float* u, int32_t on_device);

/* Populations f_i - w_i of member 0 in FP32, layout [19][N], as they stand
 * before the next collision (wall and face values included). */
ibl_status ibl_read_populations(ibl_ctx* ctx, float* g, int32_t on_device);

/* Capsule id of member 0: FP64 diagnostics and (optional) vertices[3 nv]. */
ibl_status ibl_read_capsule(ibl_ctx* ctx, int32_t id, ibl_capsule_stats* stats,
                            double* verts_out);

/* FP64 diagnostics of all n capsules of member `member` (n must equal the
 * member's capsule count), computed on the device and read back in one copy
 * of 18 doubles per capsule: the same quantities as ibl_read_capsule (volume
 * moments from the tetrahedra fanned from each capsule's first vertex; the
 * largest stretch divides by the FP32 rest lengths of the damage rule). */
ibl_status ibl_read_capsules(ibl_ctx* ctx, int32_t member, ibl_capsule_stats* stats, int32_t n);

/* Per-vertex state of a capsule of member 0: positions x(t) and x(t-dt),
 * velocity, and the total force of the last step (FP64, 3 per vertex, each
 * pointer may be NULL). */
ibl_status ibl_read_capsule_state(ibl_ctx* ctx, int32_t id, double* x, double* x_prev,
                                  double* vel, double* force);

/* Batched sweep: a new context holding copies of the (not yet stepped)
 * members' set-up, stepped together in one launch per kernel.  All members
 * must use the same storage. The member contexts stay valid. */
ibl_status ibl_ensemble_create(ibl_ctx* const* members, int32_t n, void* cuda_stream,
                               ibl_ctx** out);
int32_t ibl_num_members(const ibl_ctx* ctx);
ibl_status ibl_member_read_fields(ibl_ctx* ctx, int32_t member, float* rho, float* u,
                                  int32_t on_device);
ibl_status ibl_member_read_populations(ibl_ctx* ctx, int32_t member, float* g, int32_t on_device);
ibl_status ibl_member_read_capsule(ibl_ctx* ctx, int32_t member, int32_t id,
                                   ibl_capsule_stats* stats, double* verts_out);
ibl_status ibl_member_steps(const ibl_ctx* ctx, int32_t member, int32_t* steps_done);

/* Launch shape of the lattice kernel: threads per block (a multiple of 32, at
 * most 128, the bound the kernel is compiled for; one warp per group of 32
 * fluid nodes) and blocks per SM of a persistent grid (0 = one block per
 * threads/32 groups).  Used by the autotuner; takes effect at the next step. */
ibl_status ibl_set_launch(ibl_ctx* ctx, int32_t threads, int32_t blocks_per_sm);

/* Which form of the lattice step (Eq. evoleq with Eqs. eqfunc and forcing:
 * BGK collision and AA-pattern stream) runs over the interior fluid nodes.
 * staged = 0 (the default): the register-gather kernel, every lane loading
 * its node's 19 populations.  staged = 1: in a context holding ONE lattice,
 * every run of consecutive interior fluid nodes is cut into chunks of at
 * most 128 nodes, and each chunk's populations and tags are fetched into
 * shared memory by bulk copies (one per population span, 16-byte aligned)
 * several chunks ahead of its collision; wrap-plane nodes, batched contexts
 * and steps that record an adjoint tape keep the register kernel.  Both
 * compute the same values in the same order (bit-identical populations).
 * The staged form is measured slower on GB300 (0.26 against 0.12 ms on the
 * 512x192x128 duct with 64 capsules) and is kept as an alternative.
 * Takes effect at the next step.  IBL_ERR_ARG unless staged is 0 or 1.  A
 * staged step whose bounded wait for a copy gives up (about one second)
 * makes ibl_step return IBL_ERR_TIMEOUT. */
ibl_status ibl_set_lattice_path(ibl_ctx* ctx, int32_t staged);

/* The form the next regular step of a set-up context uses: 1 staged, 0
 * register gathers, -1 when the context is not set up yet (no step, read
 * or save has run). */
int32_t ibl_lattice_path(const ibl_ctx* ctx);

/* Autotuner of the lattice kernel's launch shape: times `steps` steps of the
 * context for each block size (32, 64, 128 threads) and persistent-grid
 * setting (blocks_per_sm 0, 1, 2, 4, 8, 16), restoring the state after every
 * trial, and keeps the fastest.  The trials are timed with CUDA events around
 * the lattice kernels; the context's state and step count are as before the
 * call.  Allocates a device snapshot of the state for the duration of the
 * call.  Outputs may be NULL. */
ibl_status ibl_autotune(ibl_ctx* ctx, int32_t steps, int32_t* threads_out,
                        int32_t* blocks_per_sm_out, double* lattice_ms_out);

/* Device time of the last ibl_step's kernels by kind, in milliseconds, when
 * timing was enabled with ibl_enable_timing (0 otherwise):
 * out[0] lattice, out[1] walls and faces, out[2] IB pass (geometry, shell,
 * marker and probe stencils), out[3] structure (repulsion, hinges, update).
 * With timing on, the steps run without CUDA graphs and every phase runs
 * alone, one after another on the context's stream (without timing the
 * structure and probe kernels overlap the IB pass and the lattice step). */
ibl_status ibl_enable_timing(ibl_ctx* ctx, int32_t on);

/* Kernel launches of one regular time step: the kernel nodes of the step's
 * CUDA graph (captured by this call if it does not exist yet; do not call it
 * inside a stream capture). */
ibl_status ibl_kernels_per_step(ibl_ctx* ctx, int32_t* n);
ibl_status ibl_kernel_times(ibl_ctx* ctx, double* out4);

/* Checkpoint / restart.  ibl_save_state copies the dynamic state of every
 * lattice of ctx (populations, status, step counters, capsule vertices x(t),
 * x(t - dt), velocities and rigid-body state) into the HOST buffer buf of
 * *bytes bytes; with buf = NULL it only sets *bytes to the size needed.
 * ibl_load_state restores such a snapshot into a context set up with the same
 * lattices, storage and capsules (IBL_ERR_ARG otherwise); stepping then
 * continues exactly where the saved context was.  Both synchronise the
 * context's stream. */
ibl_status ibl_save_state(ibl_ctx* ctx, void* buf, size_t* bytes);
ibl_status ibl_load_state(ibl_ctx* ctx, const void* buf, size_t bytes);

/* Objective of the adjoint: J = sum over the fluid nodes x with
 * lo <= x < hi (user coordinates, per axis) of d . u(x) after the last step,
 * u = (sum f e + F_body/2) / rho. */
typedef struct {
    int32_t lo[3], hi[3];
    double d[3];
} ibl_objective;

/* Discrete adjoint of n_steps lattice steps (Eq. evoleq collide + stream, Eq.
 * bbouzidi wall links, Eq. extbound faces) from the current state of a
 * context holding ONE FP32 lattice without capsules (IBL_ERR_STATE otherwise).
 * The call advances the context by n_steps exactly as ibl_step does and
 * returns J at the last step (J_out) and its derivatives
 *   grad_inlet_scale = dJ/ds for velocity-face data scaled as u_w (1 + s)
 *                      (dJ/du_max = grad_inlet_scale / u_max when the inlet
 *                      profile is proportional to its peak u_max), and
 *   grad_rj          = sum over links of dJ/dq * dq (the dq of the
 *                      ibl_wall_link records, e.g. dq/d(junction radius)),
 * with the fluid/solid tags held fixed.  The forward pass keeps a copy of the
 * populations at the start of every ckpt_every-step segment but the last,
 * whose tape ((rho, u) per node, d(value)/dq per wall link, rho per face node)
 * it records directly; the reverse pass runs the last segment's adjoint steps,
 * then recomputes each earlier segment from its copy, recording its tape, and
 * runs its adjoint steps backwards.  With ckpt_every >= n_steps nothing is
 * recomputed.  The device memory,
 *   (ceil(n_steps / ckpt_every) - 1) * populations
 *   + ckpt_every * 16 B per node + 2 * 19 * 4 B per node,
 * is allocated by the first call that needs it (cudaMalloc) and kept by the
 * context, with the CUDA graphs of the segments, until ibl_destroy; a later
 * call with more checkpoints or longer segments reallocates it.
 * Outputs may be NULL; gradients are accumulated in FP64. */
ibl_status ibl_adjoint_flow(ibl_ctx* ctx, int32_t n_steps, int32_t ckpt_every,
                            const ibl_objective* obj, double* J_out,
                            double* grad_inlet_scale, double* grad_rj);

/* Discrete adjoint of n_steps coupled steps for a capsule objective: the
 * gradient of J = dJ_dD_dOffset[0] * D + dJ_dD_dOffset[1] * offset, with D
 * the Taylor deformation index of capsule 0 after the last step and offset
 * its branch offset (the y coordinate of its volume centroid less that of the
 * symmetry plane), with respect to
 *   grad_Ca   - the capillary number of the capsule (k_s0 = rho nu u_ref / Ca,
 *               u_ref held fixed; Section "Deforming bodies constitutive model"),
 *   grad_umax - the peak inlet velocity, the velocity-face data being
 *               proportional to it (dJ/ds / u_max for data scaled by (1 + s),
 *               u_max the lattice descriptor's),
 *   grad_rj   - the junction radius, through the link distances q and the dq
 *               of the ibl_wall_link records (fluid/solid tags held fixed).
 * The context must hold one FP32 lattice with exactly one soft capsule
 * (IBL_ERR_STATE otherwise).  The reverse sweep differentiates every step as
 * ibl_step computes it (Reading T1 order): the lattice (Eq. evoleq with the
 * Guo term of the IB force, Eq. bbouzidi, Eq. extbound), the MLS
 * interpolation and spreading (Eqs. uLag, l2norm, intKernel, bodyforce), the
 * membrane, volume and probe forces (Eqs. strainFor .. hydroForNu) and the
 * Verlet update (Eqs. verletPos .. verletPosC); the MLS nearest nodes,
 * supports and singular fall-backs are held at their forward choice.  The
 * call advances the context by n_steps exactly as ibl_step does.  The
 * forward pass keeps, at the start of every ckpt_every-step segment but the
 * last, a copy of the populations and of the vertex positions, previous
 * positions and velocities; the reverse pass recomputes each earlier segment
 * from its copy while recording its tape (per step: (rho, u) and the IB
 * force of every node, d(value)/dq of every link, rho of every face node, the
 * vertex positions and velocities), then runs its adjoint steps backwards.
 * Device memory, allocated by the first call that needs it (cudaMalloc) and
 * kept by the context until ibl_destroy (a later call with more checkpoints
 * or longer segments reallocates it):
 *   (ceil(n_steps / ckpt_every) - 1) * (populations + 72 B per vertex)
 *   + ckpt_every * (32 B per node + 48 B per vertex + 4 B per link and face node)
 *   + 2 * 19 * 4 B + 32 B per node + 104 B per vertex.
 * Gradients are accumulated in FP64.  Outputs may be NULL.  Returns
 * IBL_ERR_DAMAGED / IBL_ERR_NONFINITE as ibl_step does. */
ibl_status ibl_adjoint(ibl_ctx* ctx, int32_t n_steps, int32_t ckpt_every, const double* dJ_dD_dOffset,
                       double* grad_Ca, double* grad_umax, double* grad_rj);

/* Allocation-free read of member `member`'s macroscopic fields into HOST
 * buffers rho[N] and u[3N] (either may be NULL, not both); same values and
 * layout as ibl_member_read_fields with on_device = 0.  The paper has no
 * counterpart: this is a service entry for callers that may not allocate
 * device memory (a caching allocator owns the device, or the call runs in a
 * memory-capped phase).  ibl_read_fields with pageable host buffers
 * allocates a device staging buffer on its first call; this one stages
 * through a fixed static
 * device array of 4 * IBL_NOALLOC_MAX_NODES floats (16 MiB) built into the
 * library and calls no cudaMalloc / cudaFree.
 *   - Lattices of more than IBL_NOALLOC_MAX_NODES nodes are rejected with
 *     IBL_ERR_ARG (use ibl_member_read_fields).
 *   - The context must already hold its device state (stepped, initialised or
 *     read once): setting it up allocates, so otherwise IBL_ERR_STATE.  That
 *     set-up also looks up the device's copy of the static array
 *     (cudaGetSymbolAddress), which loads the library module holding it, so
 *     the array's memory is reserved while the context is set up, not by this
 *     call.
 *   - The device that was current when the context was created must be
 *     current (IBL_ERR_STATE otherwise): the array is per device.  The call
 *     synchronises its work stream.
 *   - All contexts of the process share the one array per device: calls whose
 *     GPU work overlaps (other host threads, contexts on other streams) race
 *     on it and may return each other's data.  Serialise them. */
#define IBL_NOALLOC_MAX_NODES (1 << 20)
ibl_status ibl_read_fields_noalloc(ibl_ctx* ctx, int32_t member, float* rho, float* u);

/* Slab decomposition along x (the lattice's natural data-parallel split): the
 * owned planes [x0, x1) of a slab, and the ghost planes it also holds, lo
 * below x0 and hi above x1 - 1 (0 at a non-periodic end of the box; on a
 * periodic x axis the ghost planes wrap). */
typedef struct {
    int32_t x0, x1;
    int32_t lo, hi;
} ibl_slab;

/* Host-only planner (no CUDA call): n_slabs owned ranges that tile [0, nx),
 * balanced by plane_weight[nx] (e.g. fluid nodes per plane; NULL: uniform),
 * each at least max(halo, 1) planes wide, with lo / hi = halo ghost planes on
 * every cut side (and on both sides of a periodic axis when n_slabs > 1).
 * out[n_slabs].  IBL_ERR_ARG when nx < n_slabs * max(halo, 1), n_slabs < 1,
 * halo < 0 or a weight is negative. */
ibl_status ibl_slab_plan(int32_t nx, int32_t periodic_x, int32_t n_slabs, int32_t halo, const double* plane_weight,
                         ibl_slab* out);

/* A context that steps the lattice of `whole` (one lattice, set up but never
 * stepped or read: geometry, faces, initial state, capsules) as n_slabs
 * x-slabs, each a member of one batched context holding its owned planes plus
 * `halo` ghost planes per cut side (ibl_slab_plan with fluid-node weights).  A cut face is
 * no Dirichlet face: after every step each ghost plane is overwritten by the
 * plane of the slab that owns it (all 19 slots of every node, fluid and
 * solid), one kernel for all planes.  With halo >= 4 every owned node ends
 * each step with the populations of the undivided lattice bit for bit: a
 * node's new values depend on its neighbours' old ones (streaming, 1 plane)
 * and on post-collision values two planes upstream (the quadratic wall
 * rule), which depend on slots one plane further.
 *   - Capsules: they belong to one more member, the whole lattice as the
 *     capsules see it (tags and the IB arrays of the whole box, no
 *     populations).  Its moments at each capsule's shell nodes come from the
 *     slab that owns each node; after the marker stencils, the IB force of
 *     every shell node goes to each slab that holds the node (owner and ghost
 *     copies); a damage or non-finite flag stops every slab.  The capsule
 *     calls (ibl_read_capsule, ibl_read_capsules with member 0,
 *     ibl_read_capsule_state) address these capsules.  Owned populations
 *     then match the undivided lattice to the rounding of the spreading's
 *     atomics.
 *   - ibl_read_fields / ibl_read_populations return the whole lattice
 *     (host buffers only: on_device gives IBL_ERR_ARG); the ibl_member_*
 *     readers return slab m with its ghost planes (the whole-lattice member
 *     holds no populations: IBL_ERR_ARG).
 *   - `whole` is only read; destroy it separately.  No adjoint on a slab
 *     context.
 *   - IBL_ERR_ARG for an invalid plan (see ibl_slab_plan), halo < 4 or more
 *     than 127 slabs with capsules; IBL_ERR_STATE when whole was stepped or
 *     read. */
ibl_status ibl_slab_group_create(ibl_ctx* whole, int32_t n_slabs, int32_t halo, void* cuda_stream, ibl_ctx** out);

/* The plan of a slab context: *n_slabs on entry is the capacity of out, on
 * return the slab count (0 for a context that is not cut into slabs). */
ibl_status ibl_slab_info(const ibl_ctx* ctx, int32_t* n_slabs, ibl_slab* out);

/* Marker-based tagging of a fixed wall (Section "Boundary conditions on fixed
 * bodies", Eq. qbouzidi): the wall is a triangular mesh verts[3*n_verts]
 * (FP64, lattice units) / tris[3*n_tris] (vertex indices) whose triangle
 * centroids are its markers.  On a box of nx*ny*nz nodes (periodic[3]
 * nonzero: the axis wraps; may be NULL):
 *   - a node whose cell (the unit cube centred on it: the node floor(c + 1/2)
 *     per axis) holds a marker is solid; markers off a non-periodic box are
 *     dropped;
 *   - tag_in[N] (optional, 0 fluid / 1 solid) marks nodes solid beforehand;
 *   - every node that is not solid and has a solid node at x + e_i gets the
 *     wall link (node, i) with q = |x_b - x_L| / |e_i|, x_L the marker of the
 *     solid cell nearest to x_b, 1/2 when that cell holds no marker, clipped
 *     to [1e-6, 1] and rounded to FP32 once (distances in FP64).
 * Outputs go to HOST buffers: tag_out[N] and the links in (node, direction)
 * order as link_node / link_dir / link_q.  *n_links is the capacity of the
 * link buffers on entry and the link count on return; with all three link
 * pointers NULL the call only counts (and fills tag_out).  IBL_ERR_ARG when a
 * triangle index is out of range, a dimension is < 1, the box exceeds
 * 2^32/19 nodes, or the link buffers are missing or too small (*n_links then
 * holds the count).  The work runs on cuda_stream (NULL: the legacy stream)
 * in temporary device buffers freed before the call returns; the call
 * synchronises that stream.  Not tied to a context: its output feeds
 * ibl_set_geometry (with dq = 0). */
ibl_status ibl_voxelise_markers(const double* verts, int32_t n_verts, const int32_t* tris, int32_t n_tris,
                                int32_t nx, int32_t ny, int32_t nz, const int32_t* periodic,
                                const uint8_t* tag_in, uint8_t* tag_out, uint32_t* link_node,
                                uint32_t* link_dir, float* link_q, int64_t* n_links, void* cuda_stream);

/* Message of the last failed call on ctx (or of the last failed ibl_create /
 * ibl_ensemble_create when ctx is NULL). */
const char* ibl_last_error(const ibl_ctx* ctx);

void ibl_destroy(ibl_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* IBL_H */
