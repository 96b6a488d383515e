"""Thin ctypes binding of libibl (include/ibl.h): argument marshalling only.

Every step of the method runs in the CUDA library; this module converts numpy
arrays / torch tensors to pointers and status codes to exceptions.  It raises
ImportError when the library has not been built (there is no CPU fallback).
"""
from __future__ import annotations

import ctypes as C
import os
import re

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libibl.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "ibl.h")

STORAGE = {"f32": 0, "f16": 1, "bf16": 2}
FACE_NONE, FACE_VELOCITY, FACE_PRESSURE = 0, 1, 2

OK, ERR_ARG, ERR_OOM, ERR_CUDA, ERR_DAMAGED, ERR_NONFINITE, ERR_TIMEOUT, ERR_STATE = 0, -1, -2, -3, -4, -5, -6, -7
STATUS_NAMES = {0: "IBL_OK", -1: "IBL_ERR_ARG", -2: "IBL_ERR_OOM", -3: "IBL_ERR_CUDA", -4: "IBL_ERR_DAMAGED",
                -5: "IBL_ERR_NONFINITE", -6: "IBL_ERR_TIMEOUT", -7: "IBL_ERR_STATE"}


class LatticeDesc(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("storage", C.c_int32),
                ("periodic", C.c_int32 * 3), ("reserved", C.c_int32), ("tau", C.c_double),
                ("body_force", C.c_double * 3), ("u_max", C.c_double)]


class WallLink(C.Structure):
    _fields_ = [("node", C.c_uint32), ("dir", C.c_uint32), ("q", C.c_float), ("dq", C.c_float)]


class CapsuleParams(C.Structure):
    _fields_ = [("Ca", C.c_double), ("Eb", C.c_double), ("kv", C.c_double), ("density_ratio", C.c_double),
                ("u_ref", C.c_double), ("rigid", C.c_int32), ("reserved", C.c_int32)]


class CapsuleStats(C.Structure):
    _fields_ = [("centroid", C.c_double * 3), ("volume", C.c_double), ("area", C.c_double), ("dS", C.c_double),
                ("taylor_D", C.c_double), ("max_stretch", C.c_double), ("semi_axes", C.c_double * 3),
                ("velocity", C.c_double * 3), ("damaged", C.c_int32), ("reserved", C.c_int32)]


class Slab(C.Structure):
    _fields_ = [("x0", C.c_int32), ("x1", C.c_int32), ("lo", C.c_int32), ("hi", C.c_int32)]


class Objective(C.Structure):
    _fields_ = [("lo", C.c_int32 * 3), ("hi", C.c_int32 * 3), ("d", C.c_double * 3)]


class IBLError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


_lib = None


def lib():
    """Load libibl.so (ImportError if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                          "or python -m paper_2207_06043_gb300.build")
    L = C.CDLL(LIB_PATH)
    vp, i32, sz, dbl = C.c_void_p, C.c_int32, C.c_size_t, C.c_double
    P = C.POINTER
    sig = {
        "ibl_create": ([P(LatticeDesc), vp, P(vp)], i32),
        "ibl_set_geometry": ([vp, vp, vp, sz], i32),
        "ibl_set_inlet_velocity": ([vp, i32, vp], i32),
        "ibl_set_outlet_pressure": ([vp, i32, dbl], i32),
        "ibl_init_equilibrium": ([vp, vp, vp], i32),
        "ibl_add_capsule": ([vp, vp, i32, vp, i32, vp, P(CapsuleParams), P(i32)], i32),
        "ibl_step": ([vp, i32, P(i32)], i32),
        "ibl_read_fields": ([vp, vp, vp, i32], i32),
        "ibl_read_populations": ([vp, vp, i32], i32),
        "ibl_read_capsule": ([vp, i32, P(CapsuleStats), vp], i32),
        "ibl_read_capsule_state": ([vp, i32, vp, vp, vp, vp], i32),
        "ibl_read_capsules": ([vp, i32, vp, i32], i32),
        "ibl_ensemble_create": ([vp, i32, vp, P(vp)], i32),
        "ibl_num_members": ([vp], i32),
        "ibl_member_read_fields": ([vp, i32, vp, vp, i32], i32),
        "ibl_member_read_capsule": ([vp, i32, i32, P(CapsuleStats), vp], i32),
        "ibl_member_read_populations": ([vp, i32, vp, i32], i32),
        "ibl_member_steps": ([vp, i32, P(i32)], i32),
        "ibl_read_fields_noalloc": ([vp, i32, vp, vp], i32),
        "ibl_set_launch": ([vp, i32, i32], i32),
        "ibl_set_lattice_path": ([vp, i32], i32),
        "ibl_lattice_path": ([vp], i32),
        "ibl_enable_timing": ([vp, i32], i32),
        "ibl_kernels_per_step": ([vp, P(i32)], i32),
        "ibl_save_state": ([vp, vp, P(sz)], i32),
        "ibl_autotune": ([vp, i32, P(i32), P(i32), P(dbl)], i32),
        "ibl_adjoint_flow": ([vp, i32, i32, P(Objective), P(dbl), P(dbl), P(dbl)], i32),
        "ibl_adjoint": ([vp, i32, i32, P(dbl), P(dbl), P(dbl), P(dbl)], i32),
        "ibl_load_state": ([vp, vp, sz], i32),
        "ibl_kernel_times": ([vp, vp], i32),
        "ibl_voxelise_markers": ([vp, i32, vp, i32, i32, i32, i32, vp, vp, vp, vp, vp, vp, P(C.c_int64), vp],
                                 i32),
        "ibl_slab_plan": ([i32, i32, i32, i32, vp, P(Slab)], i32),
        "ibl_slab_group_create": ([vp, i32, i32, vp, P(vp)], i32),
        "ibl_slab_info": ([vp, P(i32), P(Slab)], i32),
        "ibl_last_error": ([vp], C.c_char_p),
        "ibl_destroy": ([vp], None),
    }
    for name, (args, res) in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    _lib = L
    return L


def header_functions():
    """Names of the functions declared in include/ibl.h."""
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:ibl_status|int32_t|void|const char\*)\s+(ibl_\w+)\s*\(", txt, re.M)))


def _ptr(a):
    """Pointer of a contiguous numpy array or torch tensor (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data_as(C.c_void_p)
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return C.c_void_p(a.data_ptr())
    raise TypeError(f"unsupported buffer {type(a)}")


def _current_stream():
    try:
        import torch
        if torch.cuda.is_available() and torch.cuda.is_initialized():
            return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    except Exception:
        pass
    return None


def voxelise_markers(verts, tris, shape, periodic=(False, False, False), tag_in=None):
    """ibl_voxelise_markers: tag a box of shape (nx, ny, nz) by the markers
    (triangle centroids) of a fixed wall mesh and measure the BFL q of every
    wall link to them (Eq. qbouzidi).  Returns (tag u8 (N,), links) with
    links a LINK-layout structured array (node, dir, q, dq = 0) in (node,
    direction) order, ready for Solver.set_geometry."""
    from .geometry import LINK_DTYPE
    L = lib()
    V = np.ascontiguousarray(verts, dtype=np.float64)
    T = np.ascontiguousarray(tris, dtype=np.int32)
    nx, ny, nz = (int(v) for v in shape)
    per = np.array([1 if p else 0 for p in periodic], dtype=np.int32)
    tin = None if tag_in is None else np.ascontiguousarray(tag_in, dtype=np.uint8)
    tag = np.empty(nx * ny * nz, dtype=np.uint8)
    n = C.c_int64(0)
    args = (_ptr(V), V.shape[0], _ptr(T), T.shape[0], nx, ny, nz, _ptr(per), _ptr(tin), _ptr(tag))
    st = L.ibl_voxelise_markers(*args, None, None, None, C.byref(n), _current_stream())
    if st != OK:
        raise IBLError(st, L.ibl_last_error(None).decode())
    node = np.empty(n.value, dtype=np.uint32)
    dirs = np.empty(n.value, dtype=np.uint32)
    q = np.empty(n.value, dtype=np.float32)
    st = L.ibl_voxelise_markers(*args, _ptr(node), _ptr(dirs), _ptr(q), C.byref(n), _current_stream())
    if st != OK:
        raise IBLError(st, L.ibl_last_error(None).decode())
    links = np.zeros(n.value, dtype=LINK_DTYPE)
    links["node"], links["dir"], links["q"] = node, dirs, q
    return tag, links


class Solver:
    """One context of the library: a lattice (or an ensemble of lattices) with
    its walls, faces and capsules."""

    def __init__(self, nx, ny, nz, tau, storage="f32", periodic=(False, False, False),
                 body_force=(0.0, 0.0, 0.0), u_max=0.02, stream=None, _handle=None):
        self._L = lib()
        self.shape = (int(nx), int(ny), int(nz))
        self.tau = float(tau)
        self.body_force = tuple(float(v) for v in body_force)
        if _handle is not None:
            self._h = _handle
            return
        d = LatticeDesc()
        d.nx, d.ny, d.nz = self.shape
        d.storage = STORAGE[storage] if isinstance(storage, str) else int(storage)
        for a in range(3):
            d.periodic[a] = 1 if periodic[a] else 0
            d.body_force[a] = float(body_force[a])
        d.tau = float(tau)
        d.u_max = float(u_max)
        h = C.c_void_p()
        st = self._L.ibl_create(C.byref(d), stream if stream is not None else _current_stream(), C.byref(h))
        if st != OK:
            raise IBLError(st, self._L.ibl_last_error(None).decode())
        self._h = h

    # -- plumbing ---------------------------------------------------------------
    def _check(self, st, allow=()):
        if st != OK and st not in allow:
            raise IBLError(st, self._L.ibl_last_error(self._h).decode())
        return st

    @property
    def n_nodes(self):
        return self.shape[0] * self.shape[1] * self.shape[2]

    def close(self):
        if getattr(self, "_h", None):
            self._L.ibl_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- set-up -----------------------------------------------------------------
    @classmethod
    def from_geometry(cls, geom, tau, storage="f32", body_force=(0.0, 0.0, 0.0), u_max=None, stream=None):
        s = cls(geom.nx, geom.ny, geom.nz, tau, storage, geom.periodic, body_force,
                geom.info.get("u_max", 0.02) if u_max is None else u_max, stream)
        s.set_geometry(geom.tag, geom.links)
        for face, spec in enumerate(geom.faces):
            if spec.kind == FACE_VELOCITY:
                s.set_inlet_velocity(face, spec.velocity)
            elif spec.kind == FACE_PRESSURE:
                s.set_outlet_pressure(face, spec.rho)
        return s

    def set_geometry(self, tag, links):
        tag = np.ascontiguousarray(tag, dtype=np.uint8).reshape(-1)
        if tag.size != self.n_nodes:
            raise ValueError("tag size mismatch")
        lk = np.ascontiguousarray(links)
        if lk.dtype.itemsize != C.sizeof(WallLink):
            raise ValueError("links must use the 16-byte (node u32, dir u32, q f32, dq f32) layout")
        self._check(self._L.ibl_set_geometry(self._h, _ptr(tag), _ptr(lk) if lk.size else None, lk.size))

    def set_inlet_velocity(self, face, u):
        u = np.ascontiguousarray(u, dtype=np.float32).reshape(-1)
        self._check(self._L.ibl_set_inlet_velocity(self._h, int(face), _ptr(u)))

    def set_outlet_pressure(self, face, rho):
        self._check(self._L.ibl_set_outlet_pressure(self._h, int(face), float(rho)))

    def init_equilibrium(self, rho=None, u=None):
        r = None if rho is None else np.ascontiguousarray(rho, dtype=np.float32).reshape(-1)
        v = None if u is None else np.ascontiguousarray(u, dtype=np.float32).reshape(-1)
        self._check(self._L.ibl_init_equilibrium(self._h, _ptr(r), _ptr(v)))

    def add_capsule(self, verts, tris, Ca=0.01, Eb=0.001, kv=1.0, density_ratio=1.1, u_ref=0.02,
                    rigid=False, vel0=None):
        V = np.ascontiguousarray(verts, dtype=np.float64).reshape(-1)
        T = np.ascontiguousarray(tris, dtype=np.int32).reshape(-1)
        p = CapsuleParams(float(Ca), float(Eb), float(kv), float(density_ratio), float(u_ref), 1 if rigid else 0, 0)
        v0 = None if vel0 is None else np.ascontiguousarray(vel0, dtype=np.float64)
        cid = C.c_int32()
        self._check(self._L.ibl_add_capsule(self._h, _ptr(V), V.size // 3, _ptr(T), T.size // 3, _ptr(v0),
                                            C.byref(p), C.byref(cid)))
        if not hasattr(self, "_nv"):
            self._nv = {}
        self._nv[(0, cid.value)] = V.size // 3
        return cid.value

    # -- stepping -----------------------------------------------------------------
    def step(self, n=1, allow_damage=False):
        done = C.c_int32()
        allow = (ERR_DAMAGED,) if allow_damage else ()
        st = self._check(self._L.ibl_step(self._h, int(n), C.byref(done)), allow)
        return done.value, st

    def set_launch(self, threads, blocks_per_sm=0):
        self._check(self._L.ibl_set_launch(self._h, int(threads), int(blocks_per_sm)))

    def set_lattice_path(self, staged=True):
        """Staged (bulk-copy) lattice kernel where the context allows it, or
        the register-gather kernel everywhere."""
        self._check(self._L.ibl_set_lattice_path(self._h, 1 if staged else 0))

    def lattice_path(self):
        """1 when the next regular step runs the staged lattice kernel, 0 for
        register gathers, -1 before the context is set up."""
        return int(self._L.ibl_lattice_path(self._h))

    def enable_timing(self, on=True):
        self._check(self._L.ibl_enable_timing(self._h, 1 if on else 0))

    def autotune(self, steps=4):
        """Pick the fastest lattice launch shape by timing trial steps (the
        state is restored).  Returns (threads, blocks_per_sm, lattice ms)."""
        t, b, ms = C.c_int32(0), C.c_int32(0), C.c_double(0.0)
        self._check(self._L.ibl_autotune(self._h, int(steps), C.byref(t), C.byref(b), C.byref(ms)))
        return int(t.value), int(b.value), float(ms.value)

    def adjoint_flow(self, steps, lo, hi, d, ckpt_every=100):
        """Discrete adjoint of `steps` lattice steps without capsules (the
        context advances by them): J = sum over the fluid nodes of the box
        [lo, hi) of d . u at the last step, dJ/ds for inlet velocities scaled
        by (1 + s), and sum_links dJ/dq dq.  Returns (J, dJ/ds, dJ/dr)."""
        ob = Objective((C.c_int32 * 3)(*lo), (C.c_int32 * 3)(*hi), (C.c_double * 3)(*d))
        J, gs, gr = C.c_double(0.0), C.c_double(0.0), C.c_double(0.0)
        self._check(self._L.ibl_adjoint_flow(self._h, int(steps), int(ckpt_every), C.byref(ob), C.byref(J),
                                             C.byref(gs), C.byref(gr)))
        return float(J.value), float(gs.value), float(gr.value)

    def adjoint(self, steps, dJ_dD_dOffset=(1.0, 0.0), ckpt_every=100):
        """Discrete adjoint of `steps` coupled steps for J = w_D D + w_off
        offset of capsule 0 after the last step (the context advances by
        them).  Returns (dJ/dCa, dJ/du_max, dJ/dr_j)."""
        w = (C.c_double * 2)(float(dJ_dD_dOffset[0]), float(dJ_dD_dOffset[1]))
        gc, gu, gr = C.c_double(0.0), C.c_double(0.0), C.c_double(0.0)
        self._check(self._L.ibl_adjoint(self._h, int(steps), int(ckpt_every), w, C.byref(gc), C.byref(gu),
                                        C.byref(gr)))
        return float(gc.value), float(gu.value), float(gr.value)

    def save_state(self):
        """Snapshot of the dynamic state (bytes)."""
        n = C.c_size_t(0)
        self._check(self._L.ibl_save_state(self._h, None, C.byref(n)))
        buf = np.empty(n.value, dtype=np.uint8)
        self._check(self._L.ibl_save_state(self._h, _ptr(buf), C.byref(n)))
        return buf.tobytes()

    def load_state(self, blob):
        """Restore a snapshot taken by save_state on an identical set-up."""
        buf = np.frombuffer(blob, dtype=np.uint8).copy()
        self._check(self._L.ibl_load_state(self._h, _ptr(buf), buf.size))

    def kernels_per_step(self):
        """Kernel launches of one regular time step (nodes of its CUDA graph)."""
        n = C.c_int32(0)
        self._check(self._L.ibl_kernels_per_step(self._h, C.byref(n)))
        return int(n.value)

    def kernel_times(self):
        out = np.zeros(4, dtype=np.float64)
        self._check(self._L.ibl_kernel_times(self._h, _ptr(out)))
        return dict(lattice=out[0], walls=out[1], ib=out[2], structure=out[3])

    # -- read-out -----------------------------------------------------------------
    def read_fields(self, member=None, out=None):
        """rho (N,), u (N,3) as float32 numpy arrays, or into out=(rho, u):
        device tensors, or host buffers (numpy arrays or CPU tensors; pinned
        tensors make the copy a direct DMA)."""
        if out is not None:
            rho, u = out
            dev = int(bool(getattr(rho, "is_cuda", False)))
            if dev != int(bool(getattr(u, "is_cuda", False))):
                raise ValueError("rho and u must both be on the device or both on the host")
            if member is None:
                self._check(self._L.ibl_read_fields(self._h, _ptr(rho), _ptr(u), dev))
            else:
                self._check(self._L.ibl_member_read_fields(self._h, int(member), _ptr(rho), _ptr(u), dev))
            return rho, u
        n = self.member_nodes(member)
        rho = np.empty(n, dtype=np.float32)
        u = np.empty((n, 3), dtype=np.float32)
        if member is None:
            self._check(self._L.ibl_read_fields(self._h, _ptr(rho), _ptr(u), 0))
        else:
            self._check(self._L.ibl_member_read_fields(self._h, int(member), _ptr(rho), _ptr(u), 0))
        return rho, u

    def member_nodes(self, member=None):
        if member is None or not hasattr(self, "member_shapes"):
            return self.n_nodes
        s = self.member_shapes[member]
        return s[0] * s[1] * s[2]

    def read_populations(self, member=None):
        g = np.empty((19, self.member_nodes(member)), dtype=np.float32)
        if member is None:
            self._check(self._L.ibl_read_populations(self._h, _ptr(g), 0))
        else:
            self._check(self._L.ibl_member_read_populations(self._h, int(member), _ptr(g), 0))
        return g

    def read_capsule(self, cid, member=None, with_verts=False):
        st = CapsuleStats()
        verts = None
        if with_verts:
            verts = np.empty(self._capsule_nv(cid, member) * 3, dtype=np.float64)
        if member is None:
            self._check(self._L.ibl_read_capsule(self._h, int(cid), C.byref(st), _ptr(verts)))
        else:
            self._check(self._L.ibl_member_read_capsule(self._h, int(member), int(cid), C.byref(st), _ptr(verts)))
        d = dict(centroid=np.array(st.centroid[:]), volume=st.volume, area=st.area, dS=st.dS,
                 taylor_D=st.taylor_D, max_stretch=st.max_stretch, semi_axes=np.array(st.semi_axes[:]),
                 velocity=np.array(st.velocity[:]), damaged=bool(st.damaged))
        if with_verts:
            d["verts"] = verts.reshape(-1, 3)
        return d

    def read_capsules(self, n, member=0):
        """FP64 diagnostics of the member's n capsules, computed on the device
        (one small read): a list of dicts as read_capsule returns."""
        arr = (CapsuleStats * n)()
        self._check(self._L.ibl_read_capsules(self._h, int(member), C.cast(arr, C.c_void_p), int(n)))
        return [dict(centroid=np.array(st.centroid[:]), volume=st.volume, area=st.area, dS=st.dS,
                     taylor_D=st.taylor_D, max_stretch=st.max_stretch, semi_axes=np.array(st.semi_axes[:]),
                     velocity=np.array(st.velocity[:]), damaged=bool(st.damaged)) for st in arr]

    def _capsule_nv(self, cid, member):
        return self._nv[(member or 0, cid)]

    def read_capsule_state(self, cid, nv):
        x = np.empty((nv, 3)); xp = np.empty((nv, 3)); v = np.empty((nv, 3)); F = np.empty((nv, 3))
        self._check(self._L.ibl_read_capsule_state(self._h, int(cid), _ptr(x), _ptr(xp), _ptr(v), _ptr(F)))
        return dict(x=x, x_prev=xp, vel=v, force=F)

    def member_steps(self, member):
        s = C.c_int32()
        self._check(self._L.ibl_member_steps(self._h, int(member), C.byref(s)))
        return s.value

    def num_members(self):
        return self._L.ibl_num_members(self._h)


def ensemble(solvers, stream=None):
    """One context stepping all solvers' lattices together (batched sweep)."""
    L = lib()
    arr = (C.c_void_p * len(solvers))(*[s._h for s in solvers])
    h = C.c_void_p()
    st = L.ibl_ensemble_create(arr, len(solvers), stream if stream is not None else _current_stream(), C.byref(h))
    if st != OK:
        raise IBLError(st, L.ibl_last_error(None).decode())
    e = Solver(*solvers[0].shape, solvers[0].tau, _handle=h)
    e.member_shapes = [s.shape for s in solvers]
    e._nv = {}
    for m, s in enumerate(solvers):
        for (mm, cid), nv in getattr(s, "_nv", {}).items():
            e._nv[(m, cid)] = nv
    return e


def slab_plan(nx, n_slabs, halo=4, periodic_x=False, plane_weight=None):
    """ibl_slab_plan (host only): list of (x0, x1, lo, hi) per slab."""
    L = lib()
    out = (Slab * int(n_slabs))()
    w = None if plane_weight is None else np.ascontiguousarray(plane_weight, dtype=np.float64)
    st = L.ibl_slab_plan(int(nx), 1 if periodic_x else 0, int(n_slabs), int(halo), _ptr(w), out)
    if st != OK:
        raise IBLError(st, L.ibl_last_error(None).decode())
    return [(o.x0, o.x1, o.lo, o.hi) for o in out]


def slab_group(whole, n_slabs, halo=4, stream=None):
    """ibl_slab_group_create: the lattice of `whole` (a Solver set up but not
    stepped) stepped as n_slabs x-slabs with halo exchange.  Returns a Solver
    whose read_fields / read_populations give the whole lattice; `whole`
    stays the caller's."""
    L = lib()
    h = C.c_void_p()
    st = L.ibl_slab_group_create(whole._h, int(n_slabs), int(halo),
                                 stream if stream is not None else _current_stream(), C.byref(h))
    if st != OK:
        raise IBLError(st, L.ibl_last_error(None).decode())
    g = Solver(*whole.shape, whole.tau, _handle=h)
    n = C.c_int32(int(n_slabs))
    out = (Slab * int(n_slabs))()
    g._check(L.ibl_slab_info(h, C.byref(n), out))
    g.slabs = [(o.x0, o.x1, o.lo, o.hi) for o in out[:n.value]]
    g.member_shapes = [(x1 - x0 + lo + hi, whole.shape[1], whole.shape[2]) for x0, x1, lo, hi in g.slabs]
    g._nv = dict(getattr(whole, "_nv", {}))
    return g


def capsule_objective_function():
    """torch.autograd.Function of the capsule objective: forward(params,
    build, steps, y_sym, ckpt_every) with params = tensor([Ca, u_max, r_j])
    builds a context with build(Ca, u_max, r_j) (a Solver holding one soft
    capsule, set up but not stepped), steps it and returns tensor([D, offset])
    of capsule 0 (offset = y of the volume centroid - y_sym); backward runs the
    library's discrete adjoint (ibl_adjoint) from the saved initial state with
    the incoming gradient as (dJ/dD, dJ/d offset) and returns dJ/d params.
    The derivative with respect to r_j goes through the dq of the wall links
    that build() supplies."""
    import torch

    class CapsuleObjective(torch.autograd.Function):
        @staticmethod
        def forward(ctx, params, build, steps, y_sym=0.0, ckpt_every=100):
            Ca, u_max, r_j = (float(v) for v in params.detach().cpu().tolist())
            s = build(Ca, u_max, r_j)
            s.step(0)
            state = s.save_state()
            s.step(int(steps))
            st = s.read_capsule(0)
            ctx.solver, ctx.state, ctx.steps, ctx.ckpt = s, state, int(steps), int(ckpt_every)
            return torch.tensor([st["taylor_D"], st["centroid"][1] - y_sym], dtype=torch.float64)

        @staticmethod
        def backward(ctx, grad_out):
            s = ctx.solver
            s.load_state(ctx.state)
            g = grad_out.detach().cpu().to(torch.float64).tolist()
            gc, gu, gr = s.adjoint(ctx.steps, (g[0], g[1]), ckpt_every=ctx.ckpt)
            return torch.tensor([gc, gu, gr], dtype=torch.float64), None, None, None, None

    return CapsuleObjective
