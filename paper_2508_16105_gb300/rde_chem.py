"""Thin Python binding of the C ABI in include/rde_chem.h (argument marshalling only).

Every function keeps the C name.  Arrays are torch CUDA tensors (float64 for
p, T, Y, h_hint; int32 for status, n_acc, n_rej; int64 for order); only their
device pointers cross the boundary.  All arithmetic happens in the sm_103a
library; there is no CPU fallback: if the library cannot be loaded, the import
fails with the reason.
"""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "_build", "librde_chem.so")

RDE_OK = 0
RDE_SCHED_AUTO, RDE_SCHED_PLAIN, RDE_SCHED_QUEUE, RDE_SCHED_BLOCK = 0, 1, 2, 3
RDE_LOAD_GENERIC, RDE_LOAD_REQUIRE_SPECIALIZED = 1, 2
RDE_METHOD_RODAS3, RDE_METHOD_ROS2, RDE_METHOD_EXTRAP = 0, 1, 2
RDE_KERNEL_GENERIC, RDE_KERNEL_SPECIALIZED, RDE_KERNEL_BLOCK = 0, 1, 2
CELL_STATUS = {0: "OK", 1: "MAX_SUBSTEPS", 2: "H_UNDERFLOW", 3: "BAD_STATE", 4: "LU_SINGULAR"}
ERRORS = {-1: "RDE_ERR_NULL", -2: "RDE_ERR_ARG", -3: "RDE_ERR_PARSE", -4: "RDE_ERR_INVALID",
          -5: "RDE_ERR_CUDA", -6: "RDE_ERR_UNSUPPORTED", -7: "RDE_ERR_ALIGN", -8: "RDE_ERR_WORKSPACE", -10: "RDE_ERR_COMPILE",
          -9: "RDE_ERR_NOMEM"}


class RdeError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("%s (%d): %s" % (ERRORS.get(code, "?"), code, msg))
        self.code = code


class rde_chem_options(C.Structure):
    _fields_ = [("rtol", C.c_double), ("atol", C.c_double), ("h_min", C.c_double), ("facmax", C.c_double),
                ("facmin", C.c_double), ("safety", C.c_double), ("max_substeps", C.c_int32),
                ("method", C.c_int32)]


class rde_block(C.Structure):
    _fields_ = [("p", C.c_void_p), ("T", C.c_void_p), ("Y", C.c_void_p), ("h_hint", C.c_void_p),
                ("status", C.c_void_p), ("n_acc", C.c_void_p), ("n_rej", C.c_void_p),
                ("n", C.c_int64), ("ldY", C.c_int64), ("cycles", C.c_void_p)]


class rde_chem_call(C.Structure):
    _fields_ = [("cells", rde_block), ("blocks", C.c_void_p), ("n_blocks", C.c_int32), ("schedule", C.c_int32),
                ("n_total", C.c_int64), ("dt", C.c_double), ("order", C.c_void_p),
                ("threads_per_cta", C.c_int32), ("ctas_per_sm", C.c_int32)]


class rde_adjoint_call(C.Structure):
    _fields_ = [("n", C.c_int64), ("p", C.c_void_p), ("T0", C.c_void_p), ("Y0", C.c_void_p), ("ldY", C.c_int64),
                ("dt", C.c_double), ("n_steps", C.c_void_p), ("total_steps", C.c_int64), ("gT", C.c_void_p),
                ("gY", C.c_void_p), ("gT0", C.c_void_p), ("gY0", C.c_void_p), ("g_lnA", C.c_void_p),
                ("g_E", C.c_void_p), ("status", C.c_void_p), ("workspace", C.c_void_p),
                ("workspace_bytes", C.c_size_t), ("schedule", C.c_int32)]


class rde_chem_stats(C.Structure):
    _fields_ = [("cells", C.c_int64), ("accepted", C.c_int64), ("rejected", C.c_int64), ("failed", C.c_int64),
                ("max_attempts", C.c_int64), ("reserved", C.c_int64 * 3)]


_lib = None


def library_path() -> str:
    return _LIB_PATH


def load_library(path: str | None = None):
    """Load librde_chem.so (built by paper_2508_16105_gb300.build); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _LIB_PATH
    if not os.path.exists(path):
        raise ImportError("librde_chem.so not built (%s); run paper_2508_16105_gb300.build.build_library()" % path)
    lib = C.CDLL(path)
    P, I64 = C.c_void_p, C.c_int64
    lib.rde_mech_load.argtypes = [C.c_char_p, C.c_size_t, C.c_int, C.POINTER(C.c_void_p)]
    lib.rde_mech_free.argtypes = [P]
    lib.rde_mech_info.argtypes = [P, C.POINTER(C.c_int), C.POINTER(C.c_int)]
    lib.rde_chem_default_options.argtypes = [C.POINTER(rde_chem_options)]
    lib.rde_chem_set_options.argtypes = [P, C.POINTER(rde_chem_options)]
    lib.rde_chem_get_options.argtypes = [P, C.POINTER(rde_chem_options)]
    lib.rde_chem_advance.argtypes = [P, I64, P, P, P, C.c_double, P]
    lib.rde_chem_advance_ex.argtypes = [P, C.POINTER(rde_chem_call), P]
    lib.rde_chem_advance_noalloc.argtypes = [P, C.POINTER(rde_chem_call), P]
    lib.rde_chem_get_stats.argtypes = [P, P, C.POINTER(rde_chem_stats)]
    lib.rde_chem_adjoint_workspace.argtypes = [P, I64, C.c_double]
    lib.rde_chem_adjoint_workspace.restype = C.c_size_t
    lib.rde_chem_adjoint_workspace_steps.argtypes = [P, I64, I64]
    lib.rde_chem_adjoint_workspace_steps.restype = C.c_size_t
    lib.rde_chem_adjoint_workspace_checkpointed.argtypes = [P, I64, I64]
    lib.rde_chem_adjoint_workspace_checkpointed.restype = C.c_size_t
    lib.rde_chem_advance_adjoint.argtypes = [P, I64, P, P, P, C.c_double, P, P, P, P, P, P, P, C.c_size_t, P]
    lib.rde_chem_advance_adjoint_ex.argtypes = [P, C.POINTER(rde_adjoint_call), P]
    lib.rde_selftest_adjoint_self_workspace.argtypes = [P, I64, C.c_int, C.c_int]
    lib.rde_selftest_adjoint_self_workspace.restype = C.c_size_t
    lib.rde_mech_get_arrhenius.argtypes = [P, P, P]
    lib.rde_mech_set_arrhenius.argtypes = [P, P, P]
    lib.rde_chem_kernel_info.argtypes = [P, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_size_t)]
    lib.rde_chem_kernel_variant.argtypes = [P, C.POINTER(C.c_int), C.POINTER(C.c_double)]
    lib.rde_selftest_batched_lu.argtypes = [C.c_int, I64, C.c_int, P, P, P, P]
    lib.rde_selftest_jit_compile.argtypes = [C.c_char_p, C.c_size_t, C.c_int, C.c_char_p, C.c_size_t, C.c_char_p,
                                             C.c_size_t, C.POINTER(C.c_double), C.POINTER(C.c_size_t)]
    lib.rde_chem_graph_create.argtypes = [P, C.POINTER(rde_chem_call), C.c_int, C.POINTER(C.c_void_p)]
    lib.rde_chem_graph_launch.argtypes = [P, P]
    lib.rde_chem_graph_destroy.argtypes = [P]
    lib.rde_chem_status.argtypes = [P, P, C.POINTER(C.c_int64)]
    lib.rde_strerror.argtypes = [C.c_int]
    lib.rde_strerror.restype = C.c_char_p
    lib.rde_last_error_message.argtypes = []
    lib.rde_last_error_message.restype = C.c_char_p
    _lib = lib
    return lib


def _check(rc: int):
    if rc != RDE_OK:
        raise RdeError(rc, _lib.rde_last_error_message().decode())


def _ptr(t):
    if t is None:
        return None
    return t.data_ptr() if hasattr(t, "data_ptr") else int(t)


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


def rde_strerror(code: int) -> str:
    return load_library().rde_strerror(code).decode()


def rde_mech_load(text: str, flags: int = 0) -> C.c_void_p:
    lib = load_library()
    b = text.encode()
    h = C.c_void_p()
    _check(lib.rde_mech_load(b, len(b), flags, C.byref(h)))
    return h


def rde_mech_free(h) -> None:
    _check(load_library().rde_mech_free(h))


def rde_mech_info(h):
    K, R = C.c_int(), C.c_int()
    _check(load_library().rde_mech_info(h, C.byref(K), C.byref(R)))
    return K.value, R.value


def rde_chem_default_options() -> rde_chem_options:
    o = rde_chem_options()
    _check(load_library().rde_chem_default_options(C.byref(o)))
    return o


def rde_chem_set_options(h, opts: rde_chem_options) -> None:
    _check(load_library().rde_chem_set_options(h, C.byref(opts)))


def rde_chem_get_options(h) -> rde_chem_options:
    o = rde_chem_options()
    _check(load_library().rde_chem_get_options(h, C.byref(o)))
    return o


def rde_chem_advance(h, n_cells: int, p, T, Y, dt: float, stream=None) -> None:
    _check(load_library().rde_chem_advance(h, n_cells, _ptr(p), _ptr(T), _ptr(Y), dt, _stream(stream)))


def _span(t) -> int:
    """Elements of t's storage from its first element on (what a pointer to it may reach)."""
    return t.untyped_storage().nbytes() // t.element_size() - t.storage_offset()


def make_block(p, T, Y, h_hint=None, status=None, n_acc=None, n_rej=None, n=None, ldY=None,
               cycles=None) -> rde_block:
    """A block of n cells over tensors: p, T and the per-cell outputs hold n values from
    their first element, Y holds species k of cell i at Y[k * ldY + i].  Raises ValueError
    when n or ldY would reach beyond a tensor's storage (the kernels cannot check it)."""
    n = int(T.shape[0]) if n is None else n
    ldY = (int(Y.stride(0)) if Y.dim() == 2 else n) if ldY is None else ldY
    if n > 0:
        if Y.dim() == 2 and Y.shape[1] > 1 and Y.stride(1) != 1:
            raise ValueError("Y must be species-major with unit stride along cells")
        if ldY < n:
            raise ValueError("ldY (%d) is smaller than the cell count (%d)" % (ldY, n))
        K = int(Y.shape[0]) if Y.dim() == 2 else 1
        if (K - 1) * ldY + n > _span(Y):
            raise ValueError("Y: %d species at ldY %d over %d cells reach beyond its storage" % (K, ldY, n))
        for name, t in (("p", p), ("T", T), ("h_hint", h_hint), ("status", status), ("n_acc", n_acc),
                        ("n_rej", n_rej), ("cycles", cycles)):
            if t is not None and (t.dim() != 1 or t.stride(0) != 1 or n > _span(t)):
                raise ValueError("%s must be a unit-stride vector holding at least n = %d values" % (name, n))
    return rde_block(_ptr(p), _ptr(T), _ptr(Y), _ptr(h_hint), _ptr(status), _ptr(n_acc), _ptr(n_rej), n, ldY,
                     _ptr(cycles))


def rde_chem_advance_ex(h, dt: float, cells: rde_block | None = None, blocks=None, n_blocks: int = 0,
                        n_total: int = 0, schedule: int = RDE_SCHED_AUTO, order=None, ctas_per_sm: int = 0,
                        stream=None, threads_per_cta: int = 0) -> None:
    c = rde_chem_call()
    if cells is not None:
        c.cells = cells
    c.blocks = _ptr(blocks)
    c.n_blocks = n_blocks
    c.n_total = n_total
    c.dt = dt
    c.schedule = schedule
    c.order = _ptr(order)
    c.threads_per_cta = threads_per_cta
    c.ctas_per_sm = ctas_per_sm
    _check(load_library().rde_chem_advance_ex(h, C.byref(c), _stream(stream)))


def rde_chem_advance_noalloc(h, dt: float, cells: rde_block | None = None, blocks=None, n_blocks: int = 0,
                             n_total: int = 0, schedule: int = RDE_SCHED_AUTO, order=None, ctas_per_sm: int = 0,
                             stream=None, threads_per_cta: int = 0) -> None:
    """rde_chem_advance_ex without any device allocation during the call (see the C header)."""
    c = rde_chem_call()
    if cells is not None:
        c.cells = cells
    c.blocks = _ptr(blocks)
    c.n_blocks = n_blocks
    c.n_total = n_total
    c.dt = dt
    c.schedule = schedule
    c.order = _ptr(order)
    c.threads_per_cta = threads_per_cta
    c.ctas_per_sm = ctas_per_sm
    _check(load_library().rde_chem_advance_noalloc(h, C.byref(c), _stream(stream)))


def _call(dt, cells=None, blocks=None, n_blocks=0, n_total=0, schedule=RDE_SCHED_AUTO, order=None, ctas_per_sm=0,
          threads_per_cta=0):
    c = rde_chem_call()
    if cells is not None:
        c.cells = cells
    c.blocks = _ptr(blocks)
    c.n_blocks = n_blocks
    c.n_total = n_total
    c.dt = dt
    c.schedule = schedule
    c.order = _ptr(order)
    c.threads_per_cta = threads_per_cta
    c.ctas_per_sm = ctas_per_sm
    return c


def rde_chem_graph_create(h, n_steps: int, dt: float, **call) -> C.c_void_p:
    """Executable graph of n_steps consecutive advances of the described cells."""
    c = _call(dt, **call)
    g = C.c_void_p()
    _check(load_library().rde_chem_graph_create(h, C.byref(c), n_steps, C.byref(g)))
    return g


def rde_chem_graph_launch(graph, stream=None) -> None:
    _check(load_library().rde_chem_graph_launch(graph, _stream(stream)))


def rde_chem_graph_destroy(graph) -> None:
    _check(load_library().rde_chem_graph_destroy(graph))


def rde_chem_adjoint_workspace(h, n_cells: int, dt: float) -> int:
    """Workspace bytes of the self-contained adjoint rde_chem_advance_adjoint."""
    return int(load_library().rde_chem_adjoint_workspace(h, n_cells, dt))


def rde_chem_adjoint_workspace_steps(h, n_cells: int, total_steps: int) -> int:
    """Workspace bytes of the recorded adjoint (step checkpoints) for known step counts."""
    return int(load_library().rde_chem_adjoint_workspace_steps(h, n_cells, total_steps))


def rde_chem_adjoint_workspace_checkpointed(h, n_cells: int, total_steps: int) -> int:
    """Workspace bytes with stage checkpoints (the reverse sweep then recomputes no stage)."""
    return int(load_library().rde_chem_adjoint_workspace_checkpointed(h, n_cells, total_steps))


def rde_chem_advance_adjoint(h, dt: float, p, T0, Y0, gT, gY, gT0, gY0, g_lnA, g_E, workspace, stream=None) -> None:
    """Self-contained adjoint of one step (Y0, gY, gY0 are [K, n] with row stride n)."""
    n = int(T0.shape[0])
    _check(load_library().rde_chem_advance_adjoint(h, n, _ptr(p), _ptr(T0), _ptr(Y0), dt, _ptr(gT), _ptr(gY),
                                                   _ptr(gT0), _ptr(gY0), _ptr(g_lnA), _ptr(g_E), _ptr(workspace),
                                                   int(workspace.numel()) if workspace is not None else 0,
                                                   _stream(stream)))


def rde_selftest_adjoint_self_workspace(h, n_cells: int, S: int, block: bool = False) -> int:
    """Self-checkpointing workspace laid out for exactly S checkpoints per cell (per CTA with block)."""
    return int(load_library().rde_selftest_adjoint_self_workspace(h, n_cells, S, 1 if block else 0))


def rde_chem_advance_adjoint_ex(h, dt: float, p, T0, Y0, n_steps, total_steps: int, gT, gY, gT0, gY0, g_lnA, g_E,
                                workspace, status=None, stream=None, schedule: int = 0) -> None:
    """Adjoint with the forward pass's step counts (n_steps), or without (n_steps=None)."""
    n = int(T0.shape[0])
    c = rde_adjoint_call(n, _ptr(p), _ptr(T0), _ptr(Y0), int(Y0.stride(0)) if n else 0, dt, _ptr(n_steps),
                         total_steps, _ptr(gT), _ptr(gY), _ptr(gT0), _ptr(gY0), _ptr(g_lnA), _ptr(g_E), _ptr(status),
                         _ptr(workspace), int(workspace.numel()) if workspace is not None else 0, schedule)
    _check(load_library().rde_chem_advance_adjoint_ex(h, C.byref(c), _stream(stream)))


def rde_mech_get_arrhenius(h, R: int):
    import numpy as np
    lnA, E = np.empty(R), np.empty(R)
    _check(load_library().rde_mech_get_arrhenius(h, lnA.ctypes.data, E.ctypes.data))
    return lnA, E


def rde_mech_set_arrhenius(h, lnA, E) -> None:
    import numpy as np
    lnA = np.ascontiguousarray(lnA, dtype=np.float64)
    E = np.ascontiguousarray(E, dtype=np.float64)
    _check(load_library().rde_mech_set_arrhenius(h, lnA.ctypes.data, E.ctypes.data))


def rde_selftest_jit_compile(text: str, part: int = 0) -> dict:
    """Generate and compile (not load) the specialised RODAS3 forward (part 0), adjoint
    (part 1) or ROS2 forward (part 2) kernels of a mechanism; no GPU needed."""
    b = text.encode()
    src = C.create_string_buffer(1 << 22)
    log = C.create_string_buffer(1 << 16)
    t, nb = C.c_double(), C.c_size_t()
    rc = load_library().rde_selftest_jit_compile(b, len(b), part, src, len(src), log, len(log), C.byref(t),
                                                 C.byref(nb))
    if rc != 0:
        raise RdeError(rc, log.value.decode() or _lib.rde_last_error_message().decode())
    return dict(source=src.value.decode(), seconds=t.value, cubin_bytes=nb.value, log=log.value.decode())


def rde_selftest_batched_lu(dmma: int, A, piv, info=None, stream=None) -> None:
    """In-place batched LU of A [batch, n, n] (device float64) with DMMA (1) or DFMA (0) updates."""
    batch, n = int(A.shape[0]), int(A.shape[1])
    _check(load_library().rde_selftest_batched_lu(dmma, batch, n, _ptr(A), _ptr(piv), _ptr(info), _stream(stream)))


def rde_chem_kernel_variant(h) -> tuple:
    """(RDE_KERNEL_* of the AUTO schedule, seconds the specialised kernel took to compile here)."""
    v, t = C.c_int(), C.c_double()
    _check(load_library().rde_chem_kernel_variant(h, C.byref(v), C.byref(t)))
    return v.value, t.value


def rde_chem_kernel_info(h) -> dict:
    t, f, b = C.c_int(), C.c_int(), C.c_size_t()
    _check(load_library().rde_chem_kernel_info(h, C.byref(t), C.byref(f), C.byref(b)))
    return dict(threads_per_cta=t.value, max_ctas_per_sm=f.value, shared_bytes=b.value)


def rde_chem_get_stats(h, stream=None) -> dict:
    s = rde_chem_stats()
    _check(load_library().rde_chem_get_stats(h, _stream(stream), C.byref(s)))
    return dict(cells=s.cells, accepted=s.accepted, rejected=s.rejected, failed=s.failed,
                max_attempts=s.max_attempts)


def rde_chem_status(h, stream=None) -> int:
    n = C.c_int64()
    _check(load_library().rde_chem_status(h, _stream(stream), C.byref(n)))
    return n.value


class BlockTable:
    """Device table of rde_block descriptors for per-block torch tensors (keeps them alive).

    blocks: list of dicts with tensors p, T, Y (Y is [K, ldY]) and optional h_hint,
    status, n_acc, n_rej.
    """

    def __init__(self, blocks: list, device=None):
        import torch
        self.blocks = blocks
        descs = [make_block(b["p"], b["T"], b["Y"], h_hint=b.get("h_hint"), status=b.get("status"),
                            n_acc=b.get("n_acc"), n_rej=b.get("n_rej"), n=int(b["T"].shape[0]),
                            ldY=int(b["Y"].stride(0)), cycles=b.get("cycles")) for b in blocks]
        raw = torch.frombuffer(bytearray(block_table_bytes(descs)), dtype=torch.uint8)
        self.table = raw.to(device or blocks[0]["T"].device)
        self.n_blocks = len(blocks)
        self.n_total = sum(int(b["T"].shape[0]) for b in blocks)

    def call_args(self) -> dict:
        return dict(blocks=self.table, n_blocks=self.n_blocks, n_total=self.n_total)


def block_table_bytes(blocks: list) -> bytes:
    """Pack rde_block descriptors for a device block table (copy them to device memory)."""
    arr = (rde_block * len(blocks))(*blocks)
    return bytes(arr)


class Mechanism:
    """Owning wrapper of a mechanism handle."""

    def __init__(self, text: str, rtol: float = 1e-8, atol: float = 1e-12, max_substeps: int = 100000,
                 flags: int = 0, method: int = RDE_METHOD_RODAS3):
        self.handle = rde_mech_load(text, flags)
        self.K, self.R = rde_mech_info(self.handle)
        o = rde_chem_default_options()
        o.rtol, o.atol, o.max_substeps, o.method = rtol, atol, max_substeps, method
        rde_chem_set_options(self.handle, o)

    def close(self):
        if self.handle is not None:
            rde_mech_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
