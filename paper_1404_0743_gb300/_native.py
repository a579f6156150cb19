"""ctypes binding of libpentago_gb300.so (argument marshalling only)."""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBPATH = os.path.join(_HERE, "libpentago_gb300.so")
_lock = threading.Lock()
_lib = None

PP_ERRORS = {1: "PP_EINVAL", 2: "PP_ENOMEM", 3: "PP_ETIMEOUT", 4: "PP_ECUDA", 5: "PP_ENOTINIT", 6: "PP_EIO"}


class PentagoError(RuntimeError):
    def __init__(self, code: int, message: str):
        super().__init__(f"{PP_ERRORS.get(code, code)}: {message}")
        self.code = code


class SectionDesc(ctypes.Structure):
    _fields_ = [("bw", (ctypes.c_uint8 * 2) * 4), ("dim", ctypes.c_uint16 * 4), ("offset", ctypes.c_uint64)]


class BatchOpts(ctypes.Structure):
    _fields_ = [("persistent", ctypes.c_int), ("threads_per_block", ctypes.c_int),
                ("ctas_per_sm", ctypes.c_int), ("stage_children", ctypes.c_int), ("largest_first", ctypes.c_int)]


class Super(ctypes.Structure):
    _fields_ = [("win", ctypes.c_uint64 * 4), ("notlose", ctypes.c_uint64 * 4)]


class Result(ctypes.Structure):
    _fields_ = [("req_id", ctypes.c_uint64), ("status", ctypes.c_int32), ("empty", ctypes.c_int32),
                ("submit_s", ctypes.c_double), ("admit_s", ctypes.c_double), ("done_s", ctypes.c_double),
                ("value", Super)]


class ServerStats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in ("submitted", "admitted", "completed", "launches", "queued",
                                               "max_active", "arena_free_largest")]


SECTION_DTYPE = np.dtype([("bw", np.uint8, (4, 2)), ("dim", np.uint16, (4,)), ("offset", np.uint64)])
assert SECTION_DTYPE.itemsize == ctypes.sizeof(SectionDesc) == 24

_P = ctypes.c_void_p
_I = ctypes.c_int
_U64 = ctypes.c_uint64
_SIZE = ctypes.c_size_t

_SIGNATURES = {
    "pp_init": ([], _I),
    "pp_shutdown": ([], None),
    "pp_last_error_string": ([], ctypes.c_char_p),
    "pp_launch_count": ([], _U64),
    "pp_quadrant_states": ([_I, _I, _P, _I], _I),
    "pp_slice_sections": ([_I, _P, _I, ctypes.POINTER(_U64)], _I),
    "pp_midgame_workspace_bytes": ([_I, _I, ctypes.POINTER(_SIZE)], _I),
    "pp_midgame_plan_create": ([_P, _I, _I, ctypes.POINTER(_P)], _I),
    "pp_midgame_plan_run": ([_P, _P, _SIZE, _P, _P], _I),
    "pp_midgame_plan_destroy": ([_P], None),
    "pp_midgame_plan_configure": ([_P, _P], _I),
    "pp_midgame_plan_autotune": ([_P, _P, _SIZE, _P, _P, _P], _I),
    "pp_midgame_plan_status": ([_P, _P], _I),
    "pp_selftest_barrier_timeout": ([_P, _P], _I),
    "pp_set_barrier_poll_limit": ([ctypes.c_uint32], _I),
    "pp_midgame_solve": ([_P, _I, _P, _I, _P, _SIZE, _P], _I),
    "pp_midgame_solve_host": ([_P, _I, _P, _I, _P, _SIZE, _P], _I),
    "pp_midgame_solve_noalloc": ([_P, _I, _P, _I, _P], _I),
    "pp_section_compute": ([_I, _P, _P, _P, _P], _I),
    "pp_section_compute_desc": ([_I, _P, _P, _P, _P, _P], _I),
    "pp_server_create_budget": ([_SIZE, _I, _I, ctypes.POINTER(_P)], _I),
    "pp_server_create": ([_P, _SIZE, _I, _I, ctypes.POINTER(_P)], _I),
    "pp_server_create_parity": ([_P, _SIZE, _I, _I, _I, ctypes.POINTER(_P)], _I),
    "pp_server_submit": ([_P, _U64, _U64], _I),
    "pp_server_poll": ([_P, _P, _I], _I),
    "pp_server_wait": ([_P, _I, ctypes.c_double], _I),
    "pp_server_get_stats": ([_P, _P], _I),
    "pp_server_destroy": ([_P], None),
    "pp_slice_step": ([_I, _P, _P, _P, _P, _P], _I),
    "pp_slice_plan_create": ([_I, _P, _P, _P, _P, ctypes.POINTER(_P)], _I),
    "pp_slice_plan_configure": ([_P, _P], _I),
    "pp_slice_plan_run": ([_P, _P], _I),
    "pp_slice_plan_autotune": ([_P, _P, _P], _I),
    "pp_slice_plan_destroy": ([_P], None),
    "pp_slice_plan_set_prepared": ([_P, _I], _I),
    "pp_prepare_children": ([_P, _U64, _P, _P], _I),
    "pp_prepare_children_ready": ([_I, _I, _P, _P, _U64, _P, _P], _I),
    "pp_stager_create": ([_I, _I, _P, _U64, _P, _P, _U64, _U64, _I, ctypes.POINTER(_P)], _I),
    "pp_stager_step": ([_P, _P, _P, _P, _P, ctypes.POINTER(_U64)], _I),
    "pp_stager_destroy": ([_P], None),
    "pp_super_digest": ([_P, _U64, _P, _P], _I),
    "pp_five_masks": ([_P, _I, _P, _P], _I),
    "pp_rmax": ([_P, _I, _P, _P], _I),
    "pp_midgame_plan_set_parity": ([_P, _I], _I),
    "pp_midgame_parity_workspace_bytes": ([_I, _I, ctypes.POINTER(_SIZE)], _I),
    "pp_midgame_solve_parity": ([_P, _I, _P, _I, _I, _P, _SIZE, _P], _I),
    "pp_shift": ([_P, _I, _I, _I, _P, _P], _I),
    "pp_symmetry_transform": ([_P, _I, _I, ctypes.POINTER(_I), _P, _P], _I),
    "pp_symmetry_info": ([_I, ctypes.POINTER(_I), ctypes.POINTER(_I)], _I),
    "pp_symmetry_board": ([_U64, _I, ctypes.POINTER(_U64)], _I),
    "pp_d4_slice_sections": ([_I, _P, _I, ctypes.POINTER(_U64)], _I),
    "pp_d4_slice_step": ([_I, _P, _P, _P, _P, _P], _I),
    "pp_d4_slice_plan_create": ([_I, _P, _P, _P, _P, ctypes.POINTER(_P)], _I),
    "pp_slice_children": ([_I, _I, _P, _P], _I),
    "pp_slice_step_sparse": ([_I, _I, _P, _P, _U64, _P, _P, _P, _P], _I),
    "pp_slice_plan_create_sparse": ([_I, _I, _P, _P, _U64, _P, _P, _P, ctypes.POINTER(_P)], _I),
    "pp_autotune_cache_load": ([ctypes.c_char_p, ctypes.POINTER(_I)], _I),
    "pp_autotune_cache_save": ([ctypes.c_char_p], _I),
    "pp_autotune_cache_clear": ([], _I),
    "pp_autotune_cache_stats": ([ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I)], _I),
}


def library_path() -> str:
    return _LIBPATH


def lib():
    """Load the CUDA library; raise if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(_LIBPATH):
                raise RuntimeError(
                    f"{_LIBPATH} is missing: build it with paper_1404_0743_gb300.build.build() "
                    "(there is no CPU fallback)")
            L = ctypes.CDLL(_LIBPATH)
            for name, (args, res) in _SIGNATURES.items():
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = res
            _lib = L
    return _lib


def _check(rc: int):
    if rc != 0:
        raise PentagoError(rc, lib().pp_last_error_string().decode())


def init():
    _check(lib().pp_init())


def launch_count() -> int:
    return int(lib().pp_launch_count())


def _stream(stream=None):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t):
    if t is None:
        return None
    if hasattr(t, "data_ptr"):
        return ctypes.c_void_p(t.data_ptr())
    return t.ctypes.data_as(ctypes.c_void_p)


def _check_cuda(t, name):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.is_contiguous()):
        raise ValueError(f"{name} must be a contiguous CUDA tensor")


def quadrant_states(black: int, white: int) -> np.ndarray:
    n = lib().pp_quadrant_states(black, white, None, 0)
    if n < 0:
        _check(-n)
    out = np.zeros(n, dtype=np.uint16)
    lib().pp_quadrant_states(black, white, _ptr(out), n)
    return out


def slice_sections(n: int, d4: bool = False):
    """Sections of slice n (the D4-minimal ones when d4) as a structured
    array (bw, dim, offset) and the total."""
    fn = lib().pp_d4_slice_sections if d4 else lib().pp_slice_sections
    count = fn(n, None, 0, None)
    if count < 0:
        _check(-count)
    out = np.zeros(count, dtype=SECTION_DTYPE)
    total = _U64(0)
    fn(n, _ptr(out), count, ctypes.byref(total))
    return out, int(total.value)


PP_ABSENT = 2 ** 64 - 1


def section_count(n: int, d4: bool = False) -> int:
    fn = lib().pp_d4_slice_sections if d4 else lib().pp_slice_sections
    count = fn(n, None, 0, None)
    if count < 0:
        _check(-count)
    return count


def _filter(n: int, filter, d4: bool):
    """A section filter as contiguous bytes, one per section of slice n."""
    if filter is None:
        return None
    f = np.ascontiguousarray(np.asarray(filter, dtype=np.uint8))
    if f.shape != (section_count(n, d4),):
        raise ValueError(f"filter of slice {n} needs {section_count(n, d4)} bytes, got shape {f.shape}")
    return f


def slice_children(n: int, filter=None, d4: bool = False):
    """One byte per section of slice n+1: 1 where a section of slice n kept
    by filter reads it."""
    f = _filter(n, filter, d4)
    out = np.zeros(section_count(n + 1, d4), dtype=np.uint8)
    _check(lib().pp_slice_children(n, int(d4), _ptr(f), _ptr(out)))
    return out


def compact_offsets(n: int, filter, d4: bool = False):
    """Where a step of slice n filtered by filter writes each section (its
    compact output: kept sections back to back in section order), PP_ABSENT
    for the others, and the number of values written."""
    secs, _ = slice_sections(n, d4)
    sizes = np.prod(secs["dim"].astype(np.uint64), axis=1)
    keep = _filter(n, filter, d4).astype(bool)
    offs = np.full(len(secs), PP_ABSENT, dtype=np.uint64)
    offs[keep] = np.cumsum(sizes[keep]) - sizes[keep]
    return offs, int(sizes[keep].sum())


def slice_step_sparse(n: int, in_values, in_offsets, out_values, filter=None, opts=None, stream=None, d4=False):
    """Sections of slice n (n <= 34) from sections of slice n+1 held anywhere
    in in_values ([count, 8] int64): in_offsets[i] is where section i starts,
    PP_ABSENT where it is not held."""
    _check_cuda(out_values, "out_values")
    _check_cuda(in_values, "in_values")
    offs = np.ascontiguousarray(np.asarray(in_offsets, dtype=np.uint64))
    if offs.shape != (section_count(n + 1, d4),):
        raise ValueError(f"in_offsets needs one entry per section of slice {n + 1}")
    f = _filter(n, filter, d4)
    o = BatchOpts(*(opts or (0, 0, 0, 0, 0)))
    _check(lib().pp_slice_step_sparse(n, int(d4), _ptr(in_values), _ptr(offs), in_values.shape[0], _ptr(out_values),
                                      _ptr(f), ctypes.byref(o), _stream(stream)))


def symmetry_info(sym: int):
    """(qmap, reflects) of board symmetry sym."""
    qmap = (_I * 4)()
    refl = _I(0)
    _check(lib().pp_symmetry_info(sym, qmap, ctypes.byref(refl)))
    return list(qmap), bool(refl.value)


def autotune_cache_load(path) -> int:
    """Merge an autotuner cache file; returns the entries read."""
    n = _I(0)
    _check(lib().pp_autotune_cache_load(os.fsencode(path), ctypes.byref(n)))
    return n.value


def autotune_cache_save(path):
    _check(lib().pp_autotune_cache_save(os.fsencode(path)))


def autotune_cache_clear():
    _check(lib().pp_autotune_cache_clear())


def autotune_cache_stats():
    """(entries, hits, misses) of the process-wide autotuner cache."""
    e, h, m = _I(0), _I(0), _I(0)
    _check(lib().pp_autotune_cache_stats(ctypes.byref(e), ctypes.byref(h), ctypes.byref(m)))
    return e.value, h.value, m.value


def symmetry_board(board: int, sym: int) -> int:
    out = _U64(0)
    _check(lib().pp_symmetry_board(int(board), sym, ctypes.byref(out)))
    return int(out.value)


def symmetry_transform(values, sym: int, turns, out, stream=None):
    t = (_I * 4)(*[int(x) for x in turns])
    _check(lib().pp_symmetry_transform(_ptr(values), values.shape[0], sym, t, _ptr(out), _stream(stream)))


def midgame_workspace_bytes(n: int, max_empty: int) -> int:
    b = _SIZE(0)
    _check(lib().pp_midgame_workspace_bytes(n, max_empty, ctypes.byref(b)))
    return int(b.value)


class MidgamePlan:
    """Validated boards with their descriptors on the device (C ``pp_midgame_plan``)."""

    def __init__(self, boards, max_empty: int):
        b = np.ascontiguousarray(np.asarray(boards, dtype=np.uint64))
        self.n = int(b.size)
        self.max_empty = max_empty
        h = ctypes.c_void_p()
        _check(lib().pp_midgame_plan_create(_ptr(b), self.n, max_empty, ctypes.byref(h)))
        self._h = h

    def run(self, workspace, out, stream=None):
        _check_cuda(workspace, "workspace")
        _check_cuda(out, "out")
        _check(lib().pp_midgame_plan_run(self._h, _ptr(workspace), workspace.numel() * workspace.element_size(),
                                         _ptr(out), _stream(stream)))

    def configure(self, mode: int, ctas_per_sm: int = 0):
        """mode 1 persistent cooperative launch, 2 one launch per level,
        3 CUDA graph of the level launches."""
        o = BatchOpts(mode, 0, ctas_per_sm, 0, 0)
        _check(lib().pp_midgame_plan_configure(self._h, ctypes.byref(o)))

    def autotune(self, workspace, out, stream=None):
        """Time every mode on this plan, keep the fastest; returns (mode, ctas_per_sm)."""
        o = BatchOpts()
        _check(lib().pp_midgame_plan_autotune(self._h, _ptr(workspace), workspace.numel() * workspace.element_size(),
                                              _ptr(out), _stream(stream), ctypes.byref(o)))
        return o.persistent, o.ctas_per_sm

    def set_parity(self, parity: int):
        """-1: every rotation; 0 / 1: only rotations g of that parity of
        g0+g1+g2+g3 (half-size fill tables; see parity_workspace_bytes)."""
        _check(lib().pp_midgame_plan_set_parity(self._h, parity))

    def status(self, stream=None):
        """Synchronise; raise PentagoError(PP_ETIMEOUT) if a barrier gave up."""
        _check(lib().pp_midgame_plan_status(self._h, _stream(stream)))

    def close(self):
        if getattr(self, "_h", None):
            lib().pp_midgame_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def midgame_solve(boards, out, max_empty: int, workspace, stream=None):
    """Super values of ``boards`` (int64 CUDA tensor of packed boards) into
    ``out`` (int64 CUDA tensor [n, 8])."""
    _check_cuda(boards, "boards")
    _check_cuda(out, "out")
    _check_cuda(workspace, "workspace")
    _check(lib().pp_midgame_solve(_ptr(boards), boards.numel(), _ptr(out), max_empty, _ptr(workspace),
                                  workspace.numel() * workspace.element_size(), _stream(stream)))


def midgame_solve_parity(boards, out, max_empty: int, parity: int, workspace, stream=None):
    """As midgame_solve, on one parity class of the rotations only."""
    _check_cuda(boards, "boards")
    _check_cuda(out, "out")
    _check_cuda(workspace, "workspace")
    _check(lib().pp_midgame_solve_parity(_ptr(boards), boards.numel(), _ptr(out), max_empty, parity, _ptr(workspace),
                                         workspace.numel() * workspace.element_size(), _stream(stream)))


def midgame_parity_workspace_bytes(n: int, max_empty: int) -> int:
    b = _SIZE(0)
    _check(lib().pp_midgame_parity_workspace_bytes(n, max_empty, ctypes.byref(b)))
    return int(b.value)


def midgame_solve_host(boards, out, max_empty: int, workspace, stream=None):
    """End to end from host arrays: ``boards`` (uint64/int64 host tensor or
    array), ``out`` (int64 host [n, 8]); inputs are copied in and results out."""
    _check_cuda(workspace, "workspace")
    _check(lib().pp_midgame_solve_host(_ptr(boards), int(boards.numel() if hasattr(boards, "numel") else boards.size),
                                       _ptr(out), max_empty, _ptr(workspace),
                                       workspace.numel() * workspace.element_size(), _stream(stream)))


def midgame_solve_noalloc(boards, out, max_empty: int, stream=None):
    """Midgame solve with no device allocation: scratch comes from the
    library's fixed 64 MiB device array (see pp_midgame_solve_noalloc)."""
    _check_cuda(boards, "boards")
    _check_cuda(out, "out")
    _check(lib().pp_midgame_solve_noalloc(_ptr(boards), boards.numel(), _ptr(out), max_empty, _stream(stream)))


def selftest_barrier_timeout(sync, stream=None) -> int:
    """Return code of the bounded-barrier self-test (PP_ETIMEOUT = 3 expected)."""
    _check_cuda(sync, "sync")
    return int(lib().pp_selftest_barrier_timeout(_ptr(sync), _stream(stream)))


def set_barrier_poll_limit(polls: int):
    """Polls a persistent midgame launch's grid barrier waits before it gives
    up (0 restores the default); a failure-path testing aid."""
    _check(lib().pp_set_barrier_poll_limit(int(polls)))


class Server:
    """Continuous-batching request server (C ``pp_server``).  ``arena`` is a
    CUDA tensor that holds the admitted queries' fill tables; keep it alive.
    With ``arena=None`` and ``budget`` (bytes) the library allocates the arena
    itself and frees it on close (every rotation only)."""

    def __init__(self, arena=None, max_slots: int = 256, max_empty: int = 16, parity: int = -1,
                 budget: int | None = None):
        h = ctypes.c_void_p()
        self._arena = arena
        if arena is None:
            if budget is None or parity != -1:
                raise ValueError("a server needs an arena tensor, or a budget (every rotation only)")
            _check(lib().pp_server_create_budget(int(budget), max_slots, max_empty, ctypes.byref(h)))
        else:
            _check_cuda(arena, "arena")
            _check(lib().pp_server_create_parity(_ptr(arena), arena.numel() * arena.element_size(), max_slots,
                                                 max_empty, parity, ctypes.byref(h)))
        self._h = h

    def submit(self, board: int, req_id: int):
        _check(lib().pp_server_submit(self._h, int(board) & ((1 << 64) - 1), int(req_id)))

    def poll(self, max_results: int = 1024):
        buf = (Result * max_results)()
        n = lib().pp_server_poll(self._h, buf, max_results)
        if n < 0:
            _check(-n)
        out = []
        for r in buf[:n]:
            value = np.array(list(r.value.win) + list(r.value.notlose), dtype=np.uint64)
            out.append(dict(req_id=r.req_id, status=r.status, empty=r.empty, submit_s=r.submit_s,
                            admit_s=r.admit_s, done_s=r.done_s, value=value))
        return out

    def wait(self, count: int, timeout_s: float = 60.0) -> int:
        n = lib().pp_server_wait(self._h, count, timeout_s)
        if n < 0:
            _check(-n)
        return n

    def stats(self):
        s = ServerStats()
        _check(lib().pp_server_get_stats(self._h, ctypes.byref(s)))
        return {n: int(getattr(s, n)) for n, _ in ServerStats._fields_}

    def close(self):
        if getattr(self, "_h", None):
            lib().pp_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _section_desc(desc):
    d = SectionDesc()
    for q in range(4):
        d.bw[q][0] = int(desc["bw"][q][0])
        d.bw[q][1] = int(desc["bw"][q][1])
        d.dim[q] = int(desc["dim"][q])
    try:
        d.offset = int(desc["offset"])
    except (KeyError, ValueError, IndexError):
        d.offset = 0
    return d


def section_compute(n: int, desc, children, out, stream=None, child_descs=None):
    """One section of slice n; ``children`` = 4 CUDA tensors or None.  With
    ``child_descs`` (4 section records or None) the call goes through
    pp_section_compute_desc, which checks them against the children the
    library expects."""
    d = _section_desc(desc)
    ptrs = (ctypes.c_void_p * 4)(*[(c.data_ptr() if c is not None else None) for c in children])
    _check_cuda(out, "out")
    if child_descs is None:
        _check(lib().pp_section_compute(n, ctypes.byref(d), ptrs, _ptr(out), _stream(stream)))
        return
    cds = [(_section_desc(c) if c is not None else None) for c in child_descs]
    cptrs = (ctypes.c_void_p * 4)(*[(ctypes.addressof(c) if c is not None else None) for c in cds])
    _check(lib().pp_section_compute_desc(n, ctypes.byref(d), ptrs, cptrs, _ptr(out), _stream(stream)))


def slice_step(n: int, in_values, out_values, filter=None, opts=None, stream=None, d4=False):
    """All (or the filtered) sections of slice n from slice n+1 (D4-reduced
    layouts when d4)."""
    _check_cuda(out_values, "out_values")
    f = _filter(n, filter, d4)
    o = BatchOpts(*(opts or (0, 0, 0, 0, 0)))
    fn = lib().pp_d4_slice_step if d4 else lib().pp_slice_step
    _check(fn(n, _ptr(in_values), _ptr(out_values), _ptr(f) if f is not None else None,
              ctypes.byref(o), _stream(stream)))


class SlicePlan:
    """Sections of slice n laid out once (C ``pp_slice_plan``); ``in_values``
    and ``out_values`` (CUDA tensors) are fixed at creation: keep them alive."""

    def __init__(self, n: int, in_values, out_values, filter=None, opts=None, d4=False, in_offsets=None):
        """in_offsets (n <= 34): slice n+1 held in part, as for slice_step_sparse."""
        _check_cuda(out_values, "out_values")
        self._h = None
        self._keep = (in_values, out_values)
        f = _filter(n, filter, d4)
        self._f = f
        o = BatchOpts(*(opts or (0, 0, 0, 0, 0)))
        h = ctypes.c_void_p()
        if in_offsets is not None:
            _check_cuda(in_values, "in_values")
            offs = np.ascontiguousarray(np.asarray(in_offsets, dtype=np.uint64))
            if offs.shape != (section_count(n + 1, d4),):
                raise ValueError(f"in_offsets needs one entry per section of slice {n + 1}")
            _check(lib().pp_slice_plan_create_sparse(n, int(d4), _ptr(in_values), _ptr(offs), in_values.shape[0],
                                                     _ptr(out_values), _ptr(f), ctypes.byref(o), ctypes.byref(h)))
        else:
            create = lib().pp_d4_slice_plan_create if d4 else lib().pp_slice_plan_create
            _check(create(n, _ptr(in_values), _ptr(out_values), _ptr(f) if f is not None else None,
                          ctypes.byref(o), ctypes.byref(h)))
        self._h = h

    def run(self, stream=None):
        _check(lib().pp_slice_plan_run(self._h, _stream(stream)))

    def configure(self, opts):
        o = BatchOpts(*opts)
        _check(lib().pp_slice_plan_configure(self._h, ctypes.byref(o)))

    def autotune(self, stream=None):
        o = BatchOpts()
        _check(lib().pp_slice_plan_autotune(self._h, _stream(stream), ctypes.byref(o)))
        return (o.persistent, o.threads_per_block, o.ctas_per_sm, o.stage_children, o.largest_first)

    def set_prepared(self, prepared=True):
        """The form of the plan's input: False/0 raw, True/1 prepared
        (prepare_children), 2 ready (prepare_children_ready)."""
        _check(lib().pp_slice_plan_set_prepared(self._h, int(prepared)))

    def close(self):
        if getattr(self, "_h", None):
            lib().pp_slice_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def prepare_children(values, out, n=None, stream=None):
    """Prepared child values (win slot ~rmax(~win), not-lose slot
    ~rmax(~notlose)) of ``values`` into ``out`` ([n, 8] int64 CUDA tensors;
    ``out`` may be ``values``)."""
    _check_cuda(values, "values")
    _check_cuda(out, "out")
    count = values.shape[0] if n is None else n
    if out.shape[0] < count:
        raise ValueError("out is smaller than the values")
    _check(lib().pp_prepare_children(_ptr(values), count, _ptr(out), _stream(stream)))


def prepare_children_ready(n: int, values, out, d4: bool = False, in_offsets=None, stream=None):
    """Ready child records of slice n+1 for the boards of slice n (win slot
    ~(F_c | rmax(~win)), not-lose slot ~(F_c | rmax(~notlose)), F_c the
    five-in-a-row set of slice n's mover) into ``out``, laid out like
    ``values`` ([count, 8] int64 CUDA tensors; ``out`` may be ``values``).
    ``values`` holds slice n+1 in its section layout, or with ``in_offsets``
    (one entry per section of slice n+1, PP_ABSENT where absent) the
    sections at those rows."""
    _check_cuda(values, "values")
    _check_cuda(out, "out")
    if out.shape[0] < values.shape[0]:
        raise ValueError("out is smaller than the values")
    offs = None
    if in_offsets is not None:
        offs = np.ascontiguousarray(np.asarray(in_offsets, dtype=np.uint64))
        if offs.shape != (section_count(n + 1, d4),):
            raise ValueError(f"in_offsets needs one entry per section of slice {n + 1}")
    _check(lib().pp_prepare_children_ready(n, int(d4), _ptr(values), _ptr(offs) if offs is not None else None,
                                           values.shape[0], _ptr(out), _stream(stream)))


class Stager:
    """Out-of-core steps of slice n < 35 (C ``pp_stager``): slice n+1 held in
    part on the device (``base``, a CUDA tensor [count, 8], section i at row
    ``dev_offsets[i]`` or PP_ABSENT) and in part on the host (``host[i]``, a
    pinned CPU tensor [size, 8] or None), with rows
    [stage_at, stage_at + stage_values) of ``base`` as staging room.  Keep
    ``base`` and the host tensors alive."""

    def __init__(self, n: int, base, dev_offsets, host, stage_at: int, stage_values: int,
                 prepared=False, d4: bool = False):
        _check_cuda(base, "base")
        self._h = None
        count = section_count(n + 1, d4)
        offs = np.ascontiguousarray(np.asarray(dev_offsets, dtype=np.uint64))
        if offs.shape != (count,) or len(host) != count:
            raise ValueError(f"dev_offsets and host need one entry per section of slice {n + 1}")
        ptrs = (ctypes.c_void_p * count)(*[(t.data_ptr() if t is not None else None) for t in host])
        self._keep = (base, list(host), ptrs, offs)
        h = ctypes.c_void_p()
        _check(lib().pp_stager_create(n, int(d4), _ptr(base), base.shape[0], _ptr(offs), ptrs, int(stage_at),
                                      int(stage_values), int(prepared), ctypes.byref(h)))
        self._h = h
        self.n, self.d4 = n, d4

    def step(self, out, filter=None, stream=None, copy_stream=None) -> int:
        """Sections of slice n kept by filter into out (back to back); returns
        the number of values copied from the host for it."""
        _check_cuda(out, "out")
        f = _filter(self.n, filter, self.d4)
        staged = _U64(0)
        _check(lib().pp_stager_step(self._h, _ptr(out), _ptr(f) if f is not None else None, _stream(stream),
                                    _stream(copy_stream), ctypes.byref(staged)))
        return int(staged.value)

    def close(self):
        if getattr(self, "_h", None):
            lib().pp_stager_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def super_digest(values, acc, n=None, stream=None):
    """Accumulate win/not-lose popcounts, an order-independent hash and the
    count of ``values`` ([n, 8] int64 CUDA tensor) into ``acc`` (4 int64)."""
    _check_cuda(acc, "acc")
    count = values.shape[0] if n is None else n
    _check(lib().pp_super_digest(_ptr(values), count, _ptr(acc), _stream(stream)))


def five_masks(boards, out, stream=None):
    _check(lib().pp_five_masks(_ptr(boards), boards.numel(), _ptr(out), _stream(stream)))


def rmax(values, out, stream=None):
    _check(lib().pp_rmax(_ptr(values), values.shape[0], _ptr(out), _stream(stream)))


def shift(values, q: int, u: int, out, stream=None):
    _check(lib().pp_shift(_ptr(values), values.shape[0], q, u, _ptr(out), _stream(stream)))
