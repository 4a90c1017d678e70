"""ctypes binding of ``libfr.so`` (include/fr.h): argument marshalling only.

Every step of the right-hand side runs in the library's CUDA kernels; this
module converts ``fr_inputs.Mesh`` objects and torch tensors into the C
structures and raw pointers the ABI takes.  There is no CPU fallback: if the
shared library is missing, importing this module raises.
"""

from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIBPATH = os.path.join(_HERE, "libfr.so")
# kernel-variant choices measured on B300 by fr_autotune, keyed by Solver.tuning_key()
TUNING_CACHE = os.path.join(_HERE, "tuning_b300.json")

OK, ERR_ARG, ERR_MESH, ERR_CUDA, ERR_NONFINITE, ERR_TIMEOUT, ERR_UNSUPPORTED, ERR_OOM = range(8)
EULER, NAVIER_STOKES = 0, 1
FP64, FP32, BF16X3, TF32X3 = 0, 1, 2, 3
ETYPES = {"quad": 0, "tri": 1, "hex": 2}
STATUS_NAMES = ["FR_OK", "FR_ERR_ARG", "FR_ERR_MESH", "FR_ERR_CUDA", "FR_ERR_NONFINITE",
                "FR_ERR_TIMEOUT", "FR_ERR_UNSUPPORTED", "FR_ERR_OOM"]

# names exported by libfr.so (every function declared in include/fr.h)
EXPORTS = ["fr_setup", "fr_layout", "fr_solution_points", "fr_operator", "fr_pairs", "fr_rhs",
           "fr_rhs_host", "fr_rk4", "fr_sum_weighted", "fr_sync_status", "fr_check_finite",
           "fr_last_error", "fr_destroy", "fr_version", "fr_profile_enable", "fr_profile_read",
           "fr_rk4_noalloc", "fr_adjoint_rhs", "fr_rk4_adjoint", "fr_set_option", "fr_fma_peak",
           "fr_euler", "fr_dopri5", "fr_setup_part", "fr_part_slots", "fr_rhs_parts", "fr_rk_step",
           "fr_rk4_host", "fr_autotune", "fr_get_tuning", "fr_set_tuning"]


class FRError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 8 else status}: {msg}")
        self.status = status


class Params(C.Structure):
    _fields_ = [("ndims", C.c_int32), ("order", C.c_int32), ("system", C.c_int32), ("precision", C.c_int32),
                ("gamma", C.c_double), ("mu", C.c_double), ("prandtl", C.c_double),
                ("ldg_beta", C.c_double), ("ldg_tau", C.c_double),
                ("bc_rho", C.c_double), ("bc_v", C.c_double * 3), ("bc_p", C.c_double),
                ("outflow_p", C.c_double), ("wall_cpTw", C.c_double), ("wall_v", C.c_double * 3),
                ("ref_rho", C.c_double), ("ref_p", C.c_double), ("correction", C.c_int32),
                ("wall2_v", C.c_double * 3)]

CORRECTIONS = {"dg": 0, "sd": 1, "hu": 2}


class EBlock(C.Structure):
    _fields_ = [("etype", C.c_int32), ("nnodes", C.c_int32), ("nelem", C.c_int64),
                ("nodes", C.POINTER(C.c_double))]


class MeshC(C.Structure):
    _fields_ = [("ndims", C.c_int32), ("nblocks", C.c_int32), ("blocks", C.POINTER(EBlock)),
                ("nbfaces", C.c_int64), ("bfaces", C.POINTER(C.c_int64)),
                ("nperiodic", C.c_int32), ("periodic", C.POINTER(C.c_double))]


_lib = None


def load():
    """Load libfr.so (fails loudly when it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIBPATH):
        raise ImportError(f"{LIBPATH} is missing: build it with paper_1312_1638_b300.build.build()")
    lib = C.CDLL(LIBPATH)
    vp, vpp = C.c_void_p, C.POINTER(C.c_void_p)
    lib.fr_setup.argtypes = [C.POINTER(MeshC), C.POINTER(Params), C.c_int, C.POINTER(vp)]
    lib.fr_layout.argtypes = [vp, C.c_int, C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                              C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
    lib.fr_solution_points.argtypes = [vp, C.c_int, C.POINTER(C.c_double)]
    lib.fr_operator.argtypes = [vp, C.c_int, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_int32),
                                C.POINTER(C.c_int32)]
    lib.fr_pairs.argtypes = [vp, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
    lib.fr_rhs.argtypes = [vp, vpp, vpp, vp]
    lib.fr_rhs_host.argtypes = [vp, vpp, vpp, vp]
    lib.fr_rk4.argtypes = [vp, vpp, C.c_double, C.c_int, vp]
    lib.fr_rk4_noalloc.argtypes = [vp, vpp, C.c_double, C.c_int, vp]
    lib.fr_rk_step.argtypes = [vp, vpp, C.c_double, C.c_int, vp]
    lib.fr_autotune.argtypes = [vp, vpp, C.c_int, vp]
    lib.fr_get_tuning.argtypes = [vp, C.c_char_p, C.c_int64]
    lib.fr_set_tuning.argtypes = [vp, C.c_char_p]
    lib.fr_rk4_host.argtypes = [vp, vpp, C.c_double, C.c_int, vp]
    lib.fr_adjoint_rhs.argtypes = [vp, vpp, vpp, vpp, vp]
    lib.fr_set_option.argtypes = [vp, C.c_char_p, C.c_int64]
    lib.fr_rk4_adjoint.argtypes = [vp, vpp, vpp, C.c_double, C.c_int, C.c_int, vp]
    lib.fr_sum_weighted.argtypes = [vp, vpp, C.POINTER(C.c_double), vp]
    lib.fr_sync_status.argtypes = [vp]
    lib.fr_check_finite.argtypes = [vp, vpp, vp]
    lib.fr_profile_enable.argtypes = [vp, C.c_int]
    lib.fr_profile_read.argtypes = [vp, C.POINTER(C.c_int32), C.c_char_p, C.POINTER(C.c_int64),
                                    C.POINTER(C.c_double)]
    lib.fr_last_error.argtypes = [vp]
    lib.fr_last_error.restype = C.c_char_p
    lib.fr_destroy.argtypes = [vp]
    lib.fr_destroy.restype = None
    lib.fr_version.restype = C.c_int32
    for name in EXPORTS:
        if name not in ("fr_last_error", "fr_destroy", "fr_version"):
            getattr(lib, name).restype = C.c_int
    _lib = lib
    return lib


def _ptrs(seq):
    arr = (C.c_void_p * len(seq))()
    for i, t in enumerate(seq):
        arr[i] = t if isinstance(t, int) else t.data_ptr()
    return arr


def _stream_ptr(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return C.c_void_p(torch.cuda.current_stream().cuda_stream)
        except ImportError:
            pass
        return C.c_void_p(0)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def adaptive_dopri5(step, save, restore, t_end, dt0, safety=0.9, facmin=0.2, facmax=10.0, max_steps=100000):
    """Step-size control for an embedded 5(4) pair (host logic).

    step(dt) advances the state by one DOPRI5 step and returns the scaled
    error norm of that step; save() / restore() keep and put back the state
    before a step, so that a rejected step (norm > 1) leaves no trace.  After
    each step dt is multiplied by a proportional-integral factor
    safety * err^(-0.17) * err_prev^(0.04) (accepted) or safety * err^(-1/5)
    (rejected), clamped to [facmin, facmax].  The paper names DOPRI5 without a
    controller (Sec. 3); the gains are those Hairer and Wanner recommend for
    this pair (Solving ODEs I, Sec. II.4).  Returns dict(t, accepted=[dt...],
    rejected=n)."""
    t, dt, prev = 0.0, float(dt0), 1e-4
    acc, rej = [], 0
    while t < t_end * (1 - 1e-14):
        if len(acc) + rej >= max_steps:
            raise RuntimeError(f"adaptive DOPRI5: {max_steps} steps without reaching t_end")
        h = min(dt, t_end - t)
        save()
        err = float(step(h))
        if not np.isfinite(err):
            restore()
            rej += 1
            dt = h * facmin
            continue
        if err <= 1.0:
            t += h
            acc.append(h)
            fac = safety * max(err, 1e-10) ** (-0.17) * prev ** 0.04
            prev = max(err, 1e-4)
        else:
            restore()
            rej += 1
            fac = safety * err ** (-1.0 / 5)
        dt = h * min(facmax, max(facmin, fac))
    return dict(t=t, accepted=acc, rejected=rej)


class PartitionedSolver:
    """The mesh split into nparts partitions, one context per rank, all on
    one device; rhs() runs fr_rhs_parts.  part: one partition index per element,
    block-major.  Each rank keeps its elements of every block in increasing
    global order (local_elements)."""

    def __init__(self, mesh, part, nparts, order, system="euler", precision="fp64", device=0, **params):
        self.mesh, self.nparts = mesh, nparts
        self.part = np.ascontiguousarray(part, dtype=np.int32)
        self.ranks = [Solver(mesh, order, system, precision, device, part=self.part, nparts=nparts, rank=r, **params)
                      for r in range(nparts)]
        self.lib = self.ranks[0].lib
        base = np.cumsum([0] + [b.nodes.shape[0] for b in mesh.blocks])
        self._local = [[np.nonzero(self.part[base[b]:base[b + 1]] == r)[0] for b in range(len(mesh.blocks))]
                       for r in range(nparts)]

    def local_elements(self, rank, b):
        """Global element indices (within block b) held by `rank`, in local order."""
        return self._local[rank][b]

    def rhs(self, u, r, stream=None):
        """u[p][b], r[p][b]: device state / result of rank p, block b."""
        ctxs = (C.c_void_p * self.nparts)(*[s.ctx for s in self.ranks])
        ua = [s._bufs(x) for s, x in zip(self.ranks, u)]             # kept alive for the call
        ra = [s._bufs(x) for s, x in zip(self.ranks, r)]
        U = (C.POINTER(C.c_void_p) * self.nparts)(*[C.cast(a, C.POINTER(C.c_void_p)) for a in ua])
        R = (C.POINTER(C.c_void_p) * self.nparts)(*[C.cast(a, C.POINTER(C.c_void_p)) for a in ra])
        self._keep = (ua, ra, U, R)
        st = self.lib.fr_rhs_parts(ctxs, self.nparts, U, R, _stream_ptr(stream))
        if st != OK:
            raise FRError(st, self.lib.fr_last_error(self.ranks[0].ctx).decode())

    def close(self):
        for s in self.ranks:
            s.close()


def fma_peak(device=0):
    """Measured (FP32, FP64) FMA throughput of the CUDA cores, TFLOP/s."""
    lib = load()
    f32, f64 = C.c_double(0), C.c_double(0)
    st = lib.fr_fma_peak(int(device), C.byref(f32), C.byref(f64))
    if st != OK:
        raise FRError(st, "fr_fma_peak failed")
    return f32.value, f64.value


class Solver:
    """An FR discretisation of a mesh (fr_setup) and its entry points.

    ``device=-1`` builds a host-only context (operators, points, pairs for
    inspection); any other value is the CUDA device ordinal.
    """

    def __init__(self, mesh, order, system="euler", precision="fp64", device=0, part=None, nparts=0, rank=0,
                 **params):
        lib = load()
        self.lib = lib
        self.mesh = mesh
        self.ndims = mesh.ndims
        self.nvars = mesh.ndims + 2
        self.precision = {"fp64": FP64, "fp32": FP32, "bf16x3": BF16X3, "tf32x3": TF32X3}[precision]
        self.system = {"euler": EULER, "ns": NAVIER_STOKES}[system]
        self.device = device
        p = Params()
        p.ndims, p.order, p.system, p.precision = mesh.ndims, order, self.system, self.precision
        p.gamma = params.get("gamma", 1.4)
        p.mu = params.get("mu", 0.0)
        p.prandtl = params.get("prandtl", 0.72)
        p.ldg_beta = params.get("ldg_beta", 0.5)
        p.ldg_tau = params.get("ldg_tau", 0.1)
        p.bc_rho = params.get("bc_rho", 1.0)
        for i, v in enumerate(params.get("bc_v", (1.0, 0.0, 0.0))):
            p.bc_v[i] = v
        p.bc_p = params.get("bc_p", 1.0)
        p.outflow_p = params.get("outflow_p", 1.0)
        p.wall_cpTw = params.get("wall_cpTw", 1.0)
        for i, v in enumerate(params.get("wall_v", (0.0, 0.0, 0.0))):
            p.wall_v[i] = v
        p.ref_rho = params.get("ref_rho", 0.0)
        p.ref_p = params.get("ref_p", 0.0)
        p.correction = CORRECTIONS[params.get("correction", "dg")]
        for i, v in enumerate(params.get("wall2_v", (0.0, 0.0, 0.0))):
            p.wall2_v[i] = v
        self.params = p
        self._keep = []
        blocks = (EBlock * len(mesh.blocks))()
        for i, b in enumerate(mesh.blocks):
            nodes = np.ascontiguousarray(b.nodes, dtype=np.float64)
            self._keep.append(nodes)
            blocks[i].etype = ETYPES[b.etype]
            blocks[i].nnodes = nodes.shape[1]
            blocks[i].nelem = nodes.shape[0]
            blocks[i].nodes = nodes.ctypes.data_as(C.POINTER(C.c_double))
        bf = np.ascontiguousarray(np.asarray(mesh.bfaces, np.int64).reshape(-1, 4))
        per = np.ascontiguousarray(np.asarray(mesh.periodic, np.float64).reshape(-1, mesh.ndims))
        self._keep += [bf, per]
        m = MeshC()
        m.ndims, m.nblocks, m.blocks = mesh.ndims, len(mesh.blocks), blocks
        m.nbfaces = bf.shape[0]
        m.bfaces = bf.ctypes.data_as(C.POINTER(C.c_int64))
        m.nperiodic = per.shape[0]
        m.periodic = per.ctypes.data_as(C.POINTER(C.c_double))
        ctx = C.c_void_p()
        if part is None:
            st = lib.fr_setup(C.byref(m), C.byref(p), device, C.byref(ctx))
        else:
            self.part = np.ascontiguousarray(part, dtype=np.int32)
            st = lib.fr_setup_part(C.byref(m), C.byref(p), device, self.part.ctypes.data_as(C.POINTER(C.c_int32)),
                                   int(nparts), int(rank), C.byref(ctx))
        if st != OK:
            raise FRError(st, lib.fr_last_error(None).decode())
        self.ctx = ctx
        self._keep = []

    def _check(self, st):
        if st != OK:
            raise FRError(st, self.lib.fr_last_error(self.ctx).decode())

    def part_slots(self):
        """{neighbour rank: int64 [nslots, 3] global L (block, element, flux point) per slot}."""
        nn = C.c_int32()
        self._check(self.lib.fr_part_slots(self.ctx, C.byref(nn), None, None, None))
        ranks = np.zeros(nn.value, np.int32)
        ns = np.zeros(nn.value, np.int64)
        self._check(self.lib.fr_part_slots(self.ctx, C.byref(nn), ranks.ctypes.data_as(C.POINTER(C.c_int32)),
                                           ns.ctypes.data_as(C.POINTER(C.c_int64)), None))
        keys = np.zeros((int(ns.sum()), 3), np.int64)
        self._check(self.lib.fr_part_slots(self.ctx, C.byref(nn), None, None,
                                           keys.ctypes.data_as(C.POINTER(C.c_int64))))
        out, o = {}, 0
        for q, n in zip(ranks, ns):
            out[int(q)] = keys[o:o + n]
            o += n
        return out

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.fr_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def nblocks(self):
        return len(self.mesh.blocks)

    def layout(self, b):
        nu, nf, nv = C.c_int32(), C.c_int32(), C.c_int32()
        ne, ld = C.c_int64(), C.c_int64()
        self._check(self.lib.fr_layout(self.ctx, b, C.byref(nu), C.byref(nf), C.byref(nv), C.byref(ne), C.byref(ld)))
        return dict(nupts=nu.value, nfpts=nf.value, nvars=nv.value, nelem=ne.value, ld=ld.value)

    def solution_points(self, b):
        L = self.layout(b)
        out = np.empty((self.ndims, L["nupts"], L["nelem"]))
        self._check(self.lib.fr_solution_points(self.ctx, b, out.ctypes.data_as(C.POINTER(C.c_double))))
        return out

    def operator(self, b, which):
        r, c = C.c_int32(), C.c_int32()
        self._check(self.lib.fr_operator(self.ctx, b, which, None, C.byref(r), C.byref(c)))
        out = np.empty((r.value, c.value))
        self._check(self.lib.fr_operator(self.ctx, b, which, out.ctypes.data_as(C.POINTER(C.c_double)), None, None))
        return out

    def pairs(self):
        n = C.c_int64()
        self._check(self.lib.fr_pairs(self.ctx, C.byref(n), None))
        out = np.empty((n.value, 6), np.int64)
        self._check(self.lib.fr_pairs(self.ctx, C.byref(n), out.ctypes.data_as(C.POINTER(C.c_int64))))
        return out

    # --------------------------------------------------------- device entry points
    @property
    def dtype_name(self):
        return "float64" if self.precision == FP64 else "float32"

    def alloc_state(self, b, torch_mod=None):
        import torch
        L = self.layout(b)
        dt = torch.float64 if self.precision == FP64 else torch.float32
        return torch.zeros((L["nupts"], L["nvars"], L["ld"]), dtype=dt, device=f"cuda:{self.device}")

    def pack(self, b, u_np):
        """[nupts, nvars, nelem] numpy -> padded [nupts, nvars, ld] host array."""
        L = self.layout(b)
        dt = np.float64 if self.precision == FP64 else np.float32
        out = np.zeros((L["nupts"], L["nvars"], L["ld"]), dt)
        out[:, :, :L["nelem"]] = u_np
        return out

    def _bufs(self, seq, host=False):
        """Pointer array of one state-shaped buffer per element block, each
        checked against the block's layout before any launch: shape [nupts,
        nvars, ld], the context's dtype, C-contiguous, on the context's GPU
        (host=True: in host memory, numpy or torch CPU).  The C ABI takes
        plain pointers and cannot see a wrong size or dtype, which would make
        its kernels read or write past the buffer; integers are taken as raw
        addresses, unchecked."""
        if len(seq) != self.nblocks:
            raise ValueError(f"{len(seq)} buffers for {self.nblocks} element blocks")
        if not hasattr(self, "_shapes"):
            self._shapes = [(L["nupts"], L["nvars"], L["ld"]) for L in (self.layout(b) for b in range(self.nblocks))]
        ptrs = []
        for b, t in enumerate(seq):
            if isinstance(t, int):
                ptrs.append(t)
                continue
            if isinstance(t, np.ndarray):
                shape, dt, contig, where = t.shape, str(t.dtype), t.flags.c_contiguous, "host"
                ptr = t.ctypes.data
            else:
                shape, dt, contig = tuple(t.shape), str(t.dtype).replace("torch.", ""), t.is_contiguous()
                where = "host" if t.device.type == "cpu" else (
                    "gpu" if t.device.type == "cuda" and t.device.index == self.device else str(t.device))
                ptr = t.data_ptr()
            want = "host" if host else "gpu"
            if tuple(shape) != self._shapes[b] or dt != self.dtype_name or not contig or where != want:
                raise ValueError(f"block {b}: buffer {tuple(shape)} {dt} {'contiguous' if contig else 'strided'} "
                                 f"on {where}; the context wants {self._shapes[b]} {self.dtype_name} contiguous "
                                 f"on {'the host' if host else f'cuda:{self.device}'}")
            ptrs.append(ptr)
        return _ptrs(ptrs)

    def rhs(self, u, r, stream=None):
        self._check(self.lib.fr_rhs(self.ctx, self._bufs(u), self._bufs(r), _stream_ptr(stream)))

    def rhs_host(self, u, r, stream=None):
        """u, r: lists of C-contiguous host arrays (numpy or pinned torch CPU tensors)."""
        self._check(self.lib.fr_rhs_host(self.ctx, self._bufs(u, True), self._bufs(r, True), _stream_ptr(stream)))

    def rk4(self, u, dt, nsteps, stream=None):
        self._check(self.lib.fr_rk4(self.ctx, self._bufs(u), C.c_double(dt), nsteps, _stream_ptr(stream)))

    def rk4_noalloc(self, u, dt, nsteps, stream=None):
        """fr_rk4_noalloc: nsteps RK4 steps in place without device allocations."""
        self._check(self.lib.fr_rk4_noalloc(self.ctx, self._bufs(u), C.c_double(dt), nsteps, _stream_ptr(stream)))

    def rk_step(self, u, dt, nsteps, stream=None):
        """fr_rk_step: nsteps steps of the context's Butcher-table RK scheme in place."""
        self._check(self.lib.fr_rk_step(self.ctx, self._bufs(u), C.c_double(dt), nsteps, _stream_ptr(stream)))

    def rk4_host(self, u, dt, nsteps, stream=None):
        """nsteps RK4 steps on host buffers (numpy arrays or pinned torch CPU
        tensors, layout of pack()); copies in and out inside the call."""
        self._check(self.lib.fr_rk4_host(self.ctx, self._bufs(u, True), C.c_double(dt), nsteps,
                                         _stream_ptr(stream)))

    def euler(self, u, dt, nsteps, stream=None):
        """nsteps forward Euler steps in place."""
        self._check(self.lib.fr_euler(self.ctx, self._bufs(u), C.c_double(dt), nsteps, _stream_ptr(stream)))

    def dopri5(self, u, dt, nsteps, atol=1e-6, rtol=1e-6, error=False, stream=None):
        """nsteps fixed DOPRI5 steps in place; with error=True returns the
        scaled RMS norm of the last step's embedded error estimate (synchronises)."""
        e = C.c_double(0.0)
        self._check(self.lib.fr_dopri5(self.ctx, self._bufs(u), C.c_double(dt), nsteps, C.c_double(atol),
                                       C.c_double(rtol), C.byref(e) if error else None, _stream_ptr(stream)))
        return e.value if error else None

    def dopri5_adaptive(self, u, t_end, dt0, atol=1e-6, rtol=1e-6, stream=None, **ctl):
        """Integrate u in place from 0 to t_end with error-controlled DOPRI5
        steps (see `adaptive_dopri5`); returns its record."""
        import torch
        backup = [torch.empty_like(x) for x in u]

        def step(dt):
            return self.dopri5(u, dt, 1, atol, rtol, error=True, stream=stream)

        def save():
            for b, x in zip(backup, u):
                b.copy_(x)

        def restore():
            for b, x in zip(backup, u):
                x.copy_(b)

        return adaptive_dopri5(step, save, restore, t_end, dt0, **ctl)

    def adjoint_rhs(self, u, lam, out, stream=None):
        """out = (dR/du)^T lam (Euler or Navier-Stokes; whole-mesh contexts)."""
        self._check(self.lib.fr_adjoint_rhs(self.ctx, self._bufs(u), self._bufs(lam), self._bufs(out), _stream_ptr(stream)))

    def rk4_adjoint(self, u0, lam, dt, nsteps, every=10, stream=None):
        """lam: dK/du_N on entry, dK/du0 on return (Euler or Navier-Stokes)."""
        self._check(self.lib.fr_rk4_adjoint(self.ctx, self._bufs(u0), self._bufs(lam), C.c_double(dt), nsteps, every,
                                            _stream_ptr(stream)))

    def sum_weighted(self, u, stream=None):
        out = np.zeros(self.nvars)
        self._check(self.lib.fr_sum_weighted(self.ctx, self._bufs(u), out.ctypes.data_as(C.POINTER(C.c_double)),
                                             _stream_ptr(stream)))
        return out

    def check_finite(self, u, stream=None):
        self._check(self.lib.fr_check_finite(self.ctx, self._bufs(u), _stream_ptr(stream)))

    def autotune(self, u, reps=2, stream=None):
        """Time every tensor-core kernel variant of each operator product on a
        copy of u and keep the fastest (fr_autotune); returns tuning()."""
        self._check(self.lib.fr_autotune(self.ctx, self._bufs(u), int(reps), _stream_ptr(stream)))
        return self.tuning()

    def tuning(self):
        """The context's kernel-variant choices as text (fr_get_tuning)."""
        buf = C.create_string_buffer(4096)
        self._check(self.lib.fr_get_tuning(self.ctx, buf, len(buf)))
        return buf.value.decode()

    def set_tuning(self, text):
        self._check(self.lib.fr_set_tuning(self.ctx, text.encode()))

    def tuning_key(self):
        """Key of a tuning cache entry: element types, order, system, precision."""
        ets = "+".join(b.etype for b in self.mesh.blocks)
        prec = {FP64: "fp64", FP32: "fp32", BF16X3: "bf16x3", TF32X3: "tf32x3"}[self.precision]
        sysn = "ns" if self.system == NAVIER_STOKES else "euler"
        return f"{ets}/p{self.params.order}/{sysn}/{prec}"

    def apply_tuning(self, u=None, cache=None, reps=2, stream=None):
        """Apply the cached choices for tuning_key() from the JSON file `cache`
        (default: the library's committed B300 table); without an entry, and
        given a state u, autotune and add the result to the file.  Returns
        (source, text) with source "cache", "autotuned" or "default"."""
        import json
        path = cache or TUNING_CACHE
        table = {}
        if os.path.exists(path):
            with open(path) as fh:
                table = json.load(fh)
        key = self.tuning_key()
        if key in table:
            self.set_tuning(table[key])
            return "cache", self.tuning()
        if u is None:
            return "default", self.tuning()
        text = self.autotune(u, reps, stream)
        table[key] = text
        with open(path, "w") as fh:
            json.dump(table, fh, indent=1, sort_keys=True)
        return "autotuned", text

    def set_option(self, name, value):
        self._check(self.lib.fr_set_option(self.ctx, name.encode(), int(value)))

    def profile_enable(self, on=True):
        self._check(self.lib.fr_profile_enable(self.ctx, 1 if on else 0))

    def profile_read(self):
        """{kernel name: (launches, total ms)} since the previous read."""
        nk = C.c_int32()
        self.lib.fr_profile_read(self.ctx, C.byref(nk), None, None, None)
        names = C.create_string_buffer(32 * nk.value)
        launches = (C.c_int64 * nk.value)()
        ms = (C.c_double * nk.value)()
        self._check(self.lib.fr_profile_read(self.ctx, C.byref(nk), names, launches, ms))
        out = {}
        for k in range(nk.value):
            name = names.raw[32 * k:32 * (k + 1)].split(b"\0", 1)[0].decode()
            out[name] = (int(launches[k]), float(ms[k]))
        return out

    def sync_status(self):
        return self.lib.fr_sync_status(self.ctx)
