"""CPU oracle for the tumour-database query (test infrastructure only).

The oracle is the plain definition of the query of Ezhov et al. (2022),
Section 2.3: threshold every database volume at u_T1Gd and u_FLAIR, compare
each entry's two segmentations with the patient's by the Dice coefficient,
add the two values (reported as their mean) and rank entries by
(score descending, index ascending).  It is written in plain C
(``oracle.c``) and wrapped here with numpy; see the header of ``oracle.c``
for every reading of the paper it takes.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA
library and never imports it.

Pinned functions (the pins live in ``tests/test_oracle_*.py``):
counts (from volumes and from byte masks), Dice, score, ranking,
thresholding (f32 and f16), the binary16
decoder, bit-plane unpacking, block means, L2 distance, nearest-neighbour
downsampling, count sketches and sign codes, and the reaction-diffusion
forward model of Section 2.1.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` with gcc into ``oracle/_build/liboracle.so``.

    Plain IEEE arithmetic: no fast-math, no floating-point contraction.
    OpenMP is used only to run the entry loop on several host cores.
    """
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-fno-fast-math", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        override = os.environ.get("DBQ_ORACLE_LIB")
        lib = ctypes.CDLL(override if override else build())
        P = ctypes.c_void_p
        i64, i32, u32, f32, f64 = (ctypes.c_int64, ctypes.c_int, ctypes.c_uint32,
                                   ctypes.c_float, ctypes.c_double)
        lib.oracle_f16_to_f64.argtypes = [ctypes.c_uint16]
        lib.oracle_f16_to_f64.restype = f64
        lib.oracle_dice.argtypes = [u32, u32, u32]
        lib.oracle_dice.restype = f64
        lib.oracle_score.argtypes = [u32] * 6
        lib.oracle_score.restype = f64
        lib.oracle_threshold_f32.argtypes = [P, i64, f32, f32, P]
        lib.oracle_threshold_f16.argtypes = [P, i64, f32, f32, P]
        lib.oracle_unpack_planes.argtypes = [P, i64, i64, P]
        for name in ("oracle_counts_f32", "oracle_counts_f16"):
            getattr(lib, name).argtypes = [P, i64, i64, P, f32, f32, i32, P, P]
            getattr(lib, name).restype = i32
        lib.oracle_counts_masks.argtypes = [P, i64, i64, P, i32, P, P]
        lib.oracle_counts_masks.restype = i32
        lib.oracle_rank.argtypes = [P, i64, i64, P, P]
        lib.oracle_rank.restype = i32
        lib.oracle_scores.argtypes = [P, i64, P, P]
        lib.oracle_block_mean.argtypes = [P, i32, i32, i32, i32, P]
        lib.oracle_block_mean.restype = i32
        lib.oracle_l2.argtypes = [P, P, i64]
        lib.oracle_l2.restype = f64
        lib.oracle_downsample_nn_u8.argtypes = [P, i32, i32, i32, i32, P]
        lib.oracle_downsample_nn_u8.restype = i32
        lib.oracle_num_threads.restype = i32
        lib.oracle_bf16_bits.argtypes = [f32]
        lib.oracle_bf16_bits.restype = ctypes.c_uint16
        lib.oracle_bf16_value.argtypes = [ctypes.c_uint16]
        lib.oracle_bf16_value.restype = f64
        lib.oracle_e4m3_value.argtypes = [ctypes.c_uint8]
        lib.oracle_e4m3_value.restype = f64
        lib.oracle_e4m3_code.argtypes = [f64]
        lib.oracle_e4m3_code.restype = ctypes.c_uint8
        lib.oracle_embed.argtypes = [P, i32, i32, i32, i32, P, P, P]
        lib.oracle_embed.restype = i32
        lib.oracle_splitmix64.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
        lib.oracle_splitmix64.restype = ctypes.c_uint64
        lib.oracle_sketch.argtypes = [P, i64, i32, P]
        lib.oracle_sketch.restype = i32
        lib.oracle_sign_code.argtypes = [P, i32, P]
        lib.oracle_hamming.argtypes = [P, P, i64]
        lib.oracle_hamming.restype = i64
        lib.oracle_rd_steps.argtypes = [f64, f64, f64, f64, f64]
        lib.oracle_rd_steps.restype = i64
        lib.oracle_rd_simulate.argtypes = [P, i32, i32, i32, P, f64, f64, P]
        lib.oracle_rd_simulate.restype = i64
        _lib = lib
        return lib


def _p(a: np.ndarray) -> int:
    return a.ctypes.data


def _c(a, dtype) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=dtype)


# ---------------------------------------------------------------- scalars
def f16_to_f64(h: int) -> float:
    """IEEE binary16 bit pattern -> value (the oracle's own decoder)."""
    return _load().oracle_f16_to_f64(int(h) & 0xFFFF)


def dice(inter: int, size_a: int, size_b: int) -> float:
    """Dice = 2|A n B| / (|A| + |B|); both empty -> 1 (Section 2.3)."""
    return _load().oracle_dice(inter, size_a, size_b)


def score(i1, i2, e1, e2, p1, p2) -> float:
    """(Dice_T1Gd + Dice_FLAIR) / 2 in binary64 (Section 2.3)."""
    return _load().oracle_score(i1, i2, e1, e2, p1, p2)


def num_threads() -> int:
    return _load().oracle_num_threads()


# ---------------------------------------------------------------- masks
def threshold(vol: np.ndarray, t1: float, t2: float) -> np.ndarray:
    """Segmentations [2][V] (uint8 0/1) of one volume: voxel in mask iff
    value >= t (binary32 compare).  float32 or float16 (as uint16 bits) input."""
    lib = _load()
    if vol.dtype == np.float16:
        vol = vol.view(np.uint16)
    v = int(vol.size)
    out = np.empty((2, v), dtype=np.uint8)
    if vol.dtype == np.uint16:
        a = _c(vol.reshape(-1), np.uint16)
        lib.oracle_threshold_f16(_p(a), v, np.float32(t1), np.float32(t2), _p(out))
    else:
        a = _c(vol.reshape(-1), np.float32)
        lib.oracle_threshold_f32(_p(a), v, np.float32(t1), np.float32(t2), _p(out))
    return out


def unpack_planes(planes: np.ndarray, v: int) -> np.ndarray:
    """Bit planes [2][words] uint32 (word w bit b = voxel 32w+b) -> [2][V] uint8."""
    lib = _load()
    a = _c(planes, np.uint32)
    words = a.shape[-1]
    if words * 32 < v:
        raise ValueError("planes too short for the volume")
    out = np.empty((2, v), dtype=np.uint8)
    lib.oracle_unpack_planes(_p(a), words, v, _p(out))
    return out


# ---------------------------------------------------------------- counts
def counts(db: np.ndarray, pmask: np.ndarray, t1: float, t2: float,
           nthreads: int = 0):
    """Per-entry counts for a database of volumes.

    db: [N, ...] float32 or float16 (or uint16 binary16 bits) volumes.
    pmask: patient segmentations [2][V] uint8.
    Returns (counts [N,4] uint32 = I1, I2, E1, E2;  pcount [2] uint32 = P1, P2).
    """
    lib = _load()
    n = int(db.shape[0])
    v = int(np.prod(db.shape[1:])) if db.ndim > 1 else 0
    pm = _c(pmask.reshape(2, v), np.uint8)
    out = np.zeros((n, 4), dtype=np.uint32)
    pc = np.zeros(2, dtype=np.uint32)
    if db.dtype in (np.float16, np.uint16):
        a = _c(db.view(np.uint16).reshape(n, v), np.uint16)
        lib.oracle_counts_f16(_p(a), n, v, _p(pm), np.float32(t1), np.float32(t2),
                              int(nthreads), _p(out), _p(pc))
    else:
        a = _c(db.reshape(n, v), np.float32)
        lib.oracle_counts_f32(_p(a), n, v, _p(pm), np.float32(t1), np.float32(t2),
                              int(nthreads), _p(out), _p(pc))
    return out, pc


def counts_masks(dbmask: np.ndarray, pmask: np.ndarray, nthreads: int = 0):
    """Counts for database entries given as masks [N][2][V] uint8 (0/1):
    (counts [N,4] = I1, I2, E1, E2;  pcount [2]).  Any other byte value
    raises ValueError."""
    lib = _load()
    n = int(dbmask.shape[0])
    v = int(dbmask.shape[-1])
    a = _c(dbmask.reshape(n, 2, v), np.uint8)
    pm = _c(pmask.reshape(2, v), np.uint8)
    out = np.zeros((n, 4), dtype=np.uint32)
    pc = np.zeros(2, dtype=np.uint32)
    if lib.oracle_counts_masks(_p(a), n, v, _p(pm), int(nthreads), _p(out), _p(pc)) != 0:
        raise ValueError("mask bytes must be 0 or 1")
    return out, pc


def scores(cnt: np.ndarray, pcount: np.ndarray) -> np.ndarray:
    lib = _load()
    c = _c(cnt, np.uint32)
    pc = _c(pcount, np.uint32)
    out = np.empty(c.shape[0], dtype=np.float64)
    lib.oracle_scores(_p(c), c.shape[0], _p(pc), _p(out))
    return out


def rank(sc: np.ndarray, k: int):
    """First k entries under (score desc, index asc) -> (index [k] int64, score [k])."""
    lib = _load()
    s = _c(sc, np.float64)
    idx = np.empty(k, dtype=np.int64)
    val = np.empty(k, dtype=np.float64)
    rc = lib.oracle_rank(_p(s), s.shape[0], int(k), _p(idx), _p(val))
    if rc != 0:
        raise ValueError(f"oracle_rank failed ({rc}): k={k} n={s.shape[0]}")
    return idx, val


def query(db: np.ndarray, patient: np.ndarray, t1: float, t2: float, k: int,
          nthreads: int = 0, patient_mask: np.ndarray | None = None):
    """The brute-force for-loop query (Section 2.3, baseline search).

    Returns a dict with index [k], score [k], counts [k,6] (I1,I2,E1,E2,P1,P2),
    and the full per-entry counts/scores for element-wise comparison.
    """
    pm = threshold(patient, t1, t2) if patient_mask is None else patient_mask
    cnt, pc = counts(db, pm, t1, t2, nthreads)
    sc = scores(cnt, pc)
    idx, val = rank(sc, k)
    hits = np.zeros((k, 6), dtype=np.uint32)
    hits[:, :4] = cnt[idx]
    hits[:, 4:] = pc
    return {"index": idx, "score": val, "counts": hits,
            "all_counts": cnt, "all_scores": sc, "pcount": pc}


# ---------------------------------------------------------------- embeddings
def block_mean(mask: np.ndarray, nx: int, ny: int, nz: int, f: int) -> np.ndarray:
    """f^3 block mean of one byte mask [V] -> [(nz/f)(ny/f)(nx/f)] float64."""
    lib = _load()
    m = _c(mask.reshape(-1), np.uint8)
    out = np.empty((nx // f) * (ny // f) * (nz // f), dtype=np.float64)
    if lib.oracle_block_mean(_p(m), nx, ny, nz, f, _p(out)) != 0:
        raise ValueError("grid not divisible by block size")
    return out


def bf16_bits(x: float) -> int:
    return _load().oracle_bf16_bits(np.float32(x))


def bf16_value(h: int) -> float:
    return _load().oracle_bf16_value(int(h) & 0xFFFF)


def e4m3_value(c: int) -> float:
    return _load().oracle_e4m3_value(int(c) & 0xFF)


def e4m3_code(x: float) -> int:
    return _load().oracle_e4m3_code(float(x))


def embed(mask: np.ndarray, nx: int, ny: int, nz: int, f: int = 8):
    """Prefilter embedding of one byte mask [V]: (bf16 bits [d] uint16,
    e4m3 codes [d] uint8, scale float32)."""
    lib = _load()
    m = _c(mask.reshape(-1), np.uint8)
    d = (nx // f) * (ny // f) * (nz // f)
    b = np.empty(d, dtype=np.uint16)
    q = np.empty(d, dtype=np.uint8)
    sc = np.empty(1, dtype=np.float32)
    if lib.oracle_embed(_p(m), nx, ny, nz, f, _p(b), _p(q), _p(sc)) != d:
        raise ValueError("grid not divisible by block size")
    return b, q, np.float32(sc[0])


def splitmix64(key: int, i: int) -> int:
    return _load().oracle_splitmix64(key, i)


def sketch(mask: np.ndarray, d: int = 4096) -> np.ndarray:
    """Count sketch [d] int32 of one byte mask [V] (see oracle.c)."""
    lib = _load()
    m = _c(mask.reshape(-1), np.uint8)
    out = np.empty(d, dtype=np.int32)
    if lib.oracle_sketch(_p(m), m.size, d, _p(out)) != 0:
        raise ValueError("d must be a power of two")
    return out


def sign_code(sk: np.ndarray) -> np.ndarray:
    lib = _load()
    a = _c(sk, np.int32)
    out = np.empty(a.size // 32, dtype=np.uint32)
    lib.oracle_sign_code(_p(a), a.size, _p(out))
    return out


def hamming(a: np.ndarray, b: np.ndarray) -> int:
    lib = _load()
    x = _c(a, np.uint32)
    y = _c(b, np.uint32)
    return int(lib.oracle_hamming(_p(x), _p(y), x.size))


def encode_values(vals: np.ndarray):
    """bf16 bits, e4m3 codes and the row scale of an integer-valued row,
    with the same rules as the block-mean embedding (scale = max|v| / 448)."""
    v = np.asarray(vals, dtype=np.float32)
    bf = np.array([bf16_bits(float(x)) for x in v], dtype=np.uint16)
    m = np.float32(np.max(np.abs(v))) if v.size else np.float32(0)
    s = np.float32(1.0) if m == 0 else np.float32(m / np.float32(448.0))
    q = np.array([e4m3_code(float(np.float32(x / s))) for x in v], dtype=np.uint8)
    return bf, q, s


def bf16_to_f64(bits: np.ndarray) -> np.ndarray:
    lib = _load()
    return np.array([lib.oracle_bf16_value(int(h)) for h in np.asarray(bits).reshape(-1)])


def e4m3_to_f64(codes: np.ndarray) -> np.ndarray:
    lib = _load()
    table = np.array([lib.oracle_e4m3_value(c) for c in range(256)])
    return table[np.asarray(codes, dtype=np.uint8)]


def l2(a: np.ndarray, b: np.ndarray) -> float:
    lib = _load()
    x = _c(a, np.float64)
    y = _c(b, np.float64)
    if x.shape != y.shape:
        raise ValueError("shape mismatch")
    return lib.oracle_l2(_p(x), _p(y), x.size)


def downsample_nn(mask: np.ndarray, nx: int, ny: int, nz: int, f: int) -> np.ndarray:
    """Nearest-neighbour downsampling of one byte mask by factor f."""
    lib = _load()
    m = _c(mask.reshape(-1), np.uint8)
    out = np.empty((nx // f) * (ny // f) * (nz // f), dtype=np.uint8)
    if lib.oracle_downsample_nn_u8(_p(m), nx, ny, nz, f, _p(out)) != 0:
        raise ValueError("grid not divisible by factor")
    return out


# ---------------------------------------------------------------- forward model
def rd_steps(t_end: float, d_w: float, rho: float, m_max: float, cfl: float) -> int:
    """Explicit-Euler step count n = ceil(T_end (6 D_w max(m) + rho) / cfl)."""
    return int(_load().oracle_rd_steps(t_end, d_w, rho, m_max, cfl))


def rd_simulate(tissue: np.ndarray, theta, u0: float = 1.0, cfl: float = 0.9):
    """u(T_end) [nz, ny, nx] binary64 of Eq. 1-2 for one theta =
    (x, y, z, D_w, rho, T_end) on the tissue map m [nz, ny, nx] (float32,
    Omega = {m > 0}); returns (u, steps).  See oracle.c for the scheme."""
    lib = _load()
    m = _c(tissue, np.float32)
    nz, ny, nx = m.shape
    th = _c(theta, np.float64).reshape(6)
    out = np.empty((nz, ny, nx), dtype=np.float64)
    n = lib.oracle_rd_simulate(_p(m), nx, ny, nz, _p(th), u0, cfl, _p(out))
    if n < 0:
        raise ValueError("seed outside the grid or the domain, or invalid parameters")
    return out, int(n)
