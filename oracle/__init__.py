"""CPU oracle for the pentago retrograde hot path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  The
product (``paper_1404_0743_gb300``) never imports it and shares no code with
it.

Parts (each cites the paper section it restates):

* O1 ``brute_force``: memoised negamax on explicit boards, one rotated root at
  a time (Section "Problem definition").
* O2 ``midgame``: rotation-separate retrograde over every filling of the empty
  cells, one explicit board and one int8 value per (fill, rotation)
  (Sections "Problem definition", "Abstracting over rotations", and the serial
  solver of "Open source and data").
* O3 ``section_value``: a board named by (slice, section, 4-D index) through the
  plain minimal-state lists of ``oracle.enumeration``, valued with O2
  (Section "Data layout and distribution").

Super values come back as ``numpy.uint64[8]``: words 0-3 are the win table,
4-7 the not-lose table, bit beta(g) = g0 + 4 g1 + 16 g2 + 64 g3 at word
beta >> 6, bit beta & 63.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

import numpy as np

from . import enumeration

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pentago_oracle.c")
_LIB = os.path.join(_HERE, "liboracle_pentago.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle in place with gcc (plain -O2, no arch flags)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-pthread", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            u64, i32, p64 = ctypes.c_uint64, ctypes.c_int, ctypes.POINTER(ctypes.c_uint64)
            p8 = ctypes.POINTER(ctypes.c_int8)
            L.oracle_brute_force.argtypes = [u64, i32, p64]
            L.oracle_brute_force.restype = i32
            L.oracle_midgame.argtypes = [u64, i32, i32, p64, p8]
            L.oracle_midgame.restype = i32
            L.oracle_midgame_threads.argtypes = [u64, i32, i32, p64, p8, i32]
            L.oracle_midgame_threads.restype = i32
            L.oracle_midgame_batch.argtypes = [p64, ctypes.c_int64, i32, p64, i32]
            L.oracle_midgame_batch.restype = i32
            L.oracle_has_five.argtypes = [u64, i32, i32]
            L.oracle_has_five.restype = i32
            L.oracle_rotate.argtypes = [u64, i32]
            L.oracle_rotate.restype = u64
            L.oracle_cells.argtypes = [u64, p8]
            L.oracle_cells.restype = i32
            L.oracle_pack.argtypes = [p8]
            L.oracle_pack.restype = u64
            _lib = L
    return _lib


class OracleError(RuntimeError):
    pass


def _out():
    a = np.zeros(8, dtype=np.uint64)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))


def brute_force(board: int, max_empty: int = 8) -> np.ndarray:
    """O1: super value by memoised negamax on explicit boards."""
    a, p = _out()
    rc = lib().oracle_brute_force(int(board), max_empty, p)
    if rc:
        raise OracleError(f"oracle_brute_force({board:#x}) -> {rc}")
    return a


def midgame(board: int, check: bool = False, max_empty: int = 16,
            all_values: bool = False, threads: int = 1):
    """O2: super value by rotation-separate retrograde over all fills.

    Up to 16 empty cells (the dense int8 table is 3^k x 256 bytes: 1.2, 3.7
    and 11 GB for k = 14, 15 and 16).  ``threads`` host threads share the
    fills of each level.  With ``all_values`` also returns the int8 table
    V[fill, beta] (fill index sum d_i 3^i over the root's empty cells in
    increasing cell order; rows of digit strings that are no position
    reachable from the root are 0)."""
    a, p = _out()
    V = None
    pv = None
    if all_values:
        k = sum(1 for c in cells(board) if c == 0)
        V = np.zeros((3 ** k, 256), dtype=np.int8)
        pv = V.ctypes.data_as(ctypes.POINTER(ctypes.c_int8))
    rc = lib().oracle_midgame_threads(int(board), max_empty, int(check), p, pv, int(threads))
    if rc:
        raise OracleError(f"oracle_midgame({board:#x}) -> {rc}")
    return (a, V) if all_values else a


def midgame_many(boards, threads: int | None = None, check: bool = False) -> np.ndarray:
    """O2 over many boards on host threads (ctypes releases the GIL)."""
    boards = [int(b) for b in boards]
    threads = threads or os.cpu_count() or 1
    lib()
    with ThreadPoolExecutor(max_workers=threads) as ex:
        res = list(ex.map(lambda b: midgame(b, check=check), boards))
    return np.stack(res) if res else np.zeros((0, 8), dtype=np.uint64)


def midgame_batch(boards, threads: int | None = None, max_empty: int = 16) -> np.ndarray:
    """O2 over many boards in one C call (one board per thread at a time,
    host threads started in C): [n, 8] uint64 super values."""
    b = np.ascontiguousarray(np.asarray(boards, dtype=np.uint64))
    out = np.zeros((len(b), 8), dtype=np.uint64)
    if len(b):
        rc = lib().oracle_midgame_batch(b.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), len(b), max_empty,
                                        out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                                        int(threads or os.cpu_count() or 1))
        if rc:
            raise OracleError(f"oracle_midgame_batch -> {rc}")
    return out


def section_boards(t) -> np.ndarray:
    """Every packed board of section t (counts per quadrant), in the
    section's layout order (quadrant 0's index fastest)."""
    ms = enumeration.minimal_states()
    lists = [np.asarray(ms[t[q]], dtype=np.uint64) << np.uint64(16 * q) for q in range(4)]
    grid = np.zeros(1, dtype=np.uint64)
    for q in range(4):  # grid index = i0 + d0 (i1 + d1 (i2 + d2 i3))
        grid = (grid[None, :] | lists[q][:, None]).reshape(-1) if q == 0 else \
            (lists[q][:, None] | grid[None, :]).reshape(-1)
    return grid


def has_five(board: int, beta: int, colour: int) -> bool:
    rc = lib().oracle_has_five(int(board), beta, colour)
    if rc < 0:
        raise OracleError("bad board")
    return bool(rc)


def rotate(board: int, beta: int) -> int:
    return int(lib().oracle_rotate(int(board), beta))


def cells(board: int) -> list[int]:
    c = (ctypes.c_int8 * 36)()
    if lib().oracle_cells(int(board), c):
        raise OracleError("bad board")
    return list(c)


def pack(cell_digits) -> int:
    c = (ctypes.c_int8 * 36)(*[int(x) for x in cell_digits])
    return int(lib().oracle_pack(c))


def section_value(n: int, t, index, check: bool = False) -> np.ndarray:
    """O3: super value of the board at 4-D index ``index`` of section ``t`` of
    slice n (36 - n empty cells), valued with O2."""
    board = enumeration.section_board(t, index)
    return midgame(board, check=check)


def bit(sv: np.ndarray, table: int, beta: int) -> int:
    """Bit beta of table 0 (win) or 1 (not lose) of a super value."""
    return int((int(sv[4 * table + (beta >> 6)]) >> (beta & 63)) & 1)


def beta_of(g) -> int:
    return g[0] + 4 * g[1] + 16 * g[2] + 64 * g[3]
