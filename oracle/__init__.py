"""FP64 CPU oracle for the photoionization source evaluation.

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only users.  Nothing here is imported
by the product package, and this package imports nothing from it; the two
share only the seeded input generators in ``sph_inputs``.

Contents
--------
* ``sph_oracle.c`` (built here with gcc + OpenMP): the direct FP64 quadrature
  of Eq. summation over the selected sets of Eq. summationI (Section 2.4,
  Section 3), the selection rules, the kernel of Eq. gfun and the
  equal-volume-ball self term.
* :func:`octree` (below): the octree and its interaction lists, built by a
  plain recursive split and by testing every box pair against the list
  definitions of the kernel-independent FMM (Section 2.4: "each leaf cube
  contains no more than a prescribed number of points"; near/far split of
  Eq. nearfar; the recursive far-field hierarchy).
* :func:`fft_convolution`: the same discrete sum as a zero-padded FFT
  convolution (an independent full-field cross-check).
* :func:`radial_reference`: the continuum Eq. integral for a spherically
  symmetric source reduced to a 1D integral.
* :func:`rel_l2`, :func:`e_delta`: the error measures of Eq. relativefun, and
  :func:`max_rel`, the gate's maximum relative error above a floor.

Parity status: every function here is pinned by ``tests/test_oracle_pins.py``
and ``tests/test_oracle_octree.py`` (the three error measures by hand-worked
cases, boundaries, empty and all-zero inputs included); none is "parity
unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sph_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "libsph_oracle.so")
_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile the C oracle (gcc, -O2, OpenMP, no fast-math).  Returns the .so path."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-fno-fast-math",
           "-ffp-contract=off", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            D, I, I64, P = ctypes.c_double, ctypes.c_int, ctypes.c_int64, ctypes.c_void_p
            lib.oracle_G.restype = D
            lib.oracle_G.argtypes = [D, D, D]
            lib.oracle_E1.restype = D
            lib.oracle_E1.argtypes = [D]
            lib.oracle_self_integral.restype = D
            lib.oracle_self_integral.argtypes = [D, D, D]
            lib.oracle_self_radius.restype = D
            lib.oracle_self_radius.argtypes = [D]
            lib.oracle_select.restype = I
            lib.oracle_select.argtypes = [I64, P, P, P, D, D, D, P, P, P, P]
            lib.oracle_sph.restype = I
            lib.oracle_sph.argtypes = [I, I, I, D, D, D, P, D, P, I64, P, I64, I, P]
            lib.oracle_sph_longdouble.restype = I
            lib.oracle_sph_longdouble.argtypes = [I, I, I, D, D, D, P, D, P, I64, P, I64, I, D, P]
            lib.oracle_num_threads.restype = I
            lib.oracle_set_num_threads.restype = None
            lib.oracle_set_num_threads.argtypes = [I]
            _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def alpha_beta(pO2, chi_min, chi_max):
    """alpha = chi_min*p_O2, beta = chi_max*p_O2 (cm^-1), from Eq. gfun."""
    return chi_min * pO2, chi_max * pO2


def G(R, alpha, beta):
    """Discrete kernel between distinct cells, Eq. gfun / (4 pi R^2), FP64."""
    lib = _load()
    return float(lib.oracle_G(float(R), float(alpha), float(beta)))


def E1(x):
    return float(_load().oracle_E1(float(x)))


def self_integral(h, alpha, beta):
    """Integral of G over the ball of one cell's volume (dimensionless)."""
    lib = _load()
    return float(lib.oracle_self_integral(lib.oracle_self_radius(float(h)), float(alpha), float(beta)))


def num_threads():
    return int(_load().oracle_num_threads())


def set_num_threads(n):
    """Threads of the oracle's OpenMP loops from now on (returns the previous count)."""
    prev = num_threads()
    _load().oracle_set_num_threads(int(n))
    return prev


def select(q, emag=None, mask=None, i_frac=0.0, e_frac=0.0, e_applied=0.0):
    """Source and target index sets (ascending int32), Section 3 selection rules."""
    lib = _load()
    q = np.ascontiguousarray(q, dtype=np.float32)
    n = q.size
    em = None if emag is None else np.ascontiguousarray(emag, dtype=np.float32)
    mk = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8)
    J = np.empty(n, np.int32)
    T = np.empty(n, np.int32)
    nJ = ctypes.c_int64()
    nT = ctypes.c_int64()
    lib.oracle_select(n, _ptr(q), _ptr(em), _ptr(mk), float(i_frac), float(e_frac),
                      float(e_applied), _ptr(J), ctypes.byref(nJ), _ptr(T), ctypes.byref(nT))
    return J[:nJ.value].copy(), T[:nT.value].copy()


def sph(nx, ny, nz, h, alpha, beta, q, source_scale, J, T, self_mode=1):
    """S_ph at the targets T (FP64, in T's order) from the sources J (ascending)."""
    lib = _load()
    q = np.ascontiguousarray(q, dtype=np.float32)
    J = np.ascontiguousarray(J, dtype=np.int32)
    T = np.ascontiguousarray(T, dtype=np.int32)
    assert J.size <= 1 or np.all(np.diff(J) > 0), "J must be strictly ascending"
    S = np.zeros(T.size, np.float64)
    lib.oracle_sph(int(nx), int(ny), int(nz), float(h), float(alpha), float(beta), _ptr(q),
                   float(source_scale), _ptr(J), J.size, _ptr(T), T.size, int(self_mode), _ptr(S))
    return S


def sph_longdouble(nx, ny, nz, h, alpha, beta, q, source_scale, J, T, self_mode=1, self_int=0.0):
    """Extended-precision brute force of the same sum (tiny grids only)."""
    lib = _load()
    q = np.ascontiguousarray(q, dtype=np.float32)
    J = np.ascontiguousarray(J, dtype=np.int32)
    T = np.ascontiguousarray(T, dtype=np.int32)
    S = np.zeros(T.size, np.float64)
    lib.oracle_sph_longdouble(int(nx), int(ny), int(nz), float(h), float(alpha), float(beta),
                              _ptr(q), float(source_scale), _ptr(J), J.size, _ptr(T), T.size,
                              int(self_mode), float(self_int), _ptr(S))
    return S


def sph_problem(p, J=None, T=None, self_mode=1, mask=None):
    """Convenience: oracle S_ph for a ``sph_inputs.Problem`` (selection per its criteria)."""
    a, b = alpha_beta(p.pO2_torr, p.chi_min, p.chi_max)
    if J is None or T is None:
        Js, Ts = select(p.q, None if (p.targets_all or mask is not None) else p.emag, mask,
                        p.i_frac, p.e_frac, p.e_applied)
        J = Js if J is None else J
        T = Ts if T is None else T
    return sph(p.nx, p.ny, p.nz, p.h, a, b, p.q, p.source_scale, J, T, self_mode), J, T


# ----------------------------------------------------------------------------
# Error measures of Eq. relativefun
# ----------------------------------------------------------------------------

def rel_l2(num, ref):
    """E_V / 100: ||num - ref||_2 / ||ref||_2."""
    num = np.asarray(num, np.float64)
    ref = np.asarray(ref, np.float64)
    d = np.linalg.norm(ref)
    return float(np.linalg.norm(num - ref) / d) if d > 0 else float(np.linalg.norm(num))


def rel_l2_weighted(num, ref, weight):
    """E_V / 100 of a whole set estimated from a weighted sample of it: each sampled entry
    stands for ``weight`` entries, sqrt(sum w (num - ref)^2 / sum w ref^2)."""
    num = np.asarray(num, np.float64)
    ref = np.asarray(ref, np.float64)
    w = np.broadcast_to(np.asarray(weight, np.float64), ref.shape)
    d = float(np.sum(w * ref * ref))
    e = float(np.sum(w * (num - ref) ** 2))
    return float(np.sqrt(e / d)) if d > 0 else float(np.sqrt(e))


def max_rel(num, ref, floor_frac=1e-3):
    """max |num-ref|/ref over entries with ref > floor_frac * max(ref)."""
    num = np.asarray(num, np.float64)
    ref = np.asarray(ref, np.float64)
    if ref.size == 0:
        return 0.0
    sel = ref > floor_frac * ref.max()
    if not np.any(sel):
        return 0.0
    return float(np.max(np.abs(num[sel] - ref[sel]) / ref[sel]))


def e_delta(num, ref, pts, x0, delta):
    """E_delta(x0) / 100: mean relative error over the points within ``delta`` of x0 (the
    boundary included); 0 for an empty ball.  ``ref`` must be positive inside the ball."""
    pts = np.asarray(pts, np.float64)
    sel = np.linalg.norm(pts - np.asarray(x0)[None, :], axis=1) <= delta
    if not np.any(sel):
        return 0.0
    num = np.asarray(num, np.float64)[sel]
    ref = np.asarray(ref, np.float64)[sel]
    return float(np.mean(np.abs(num - ref) / ref))


# ----------------------------------------------------------------------------
# Full-field cross-check: the discrete sum over a uniform grid is a convolution
# ----------------------------------------------------------------------------

def fft_convolution(nx, ny, nz, h, alpha, beta, q, source_scale, J, self_mode=1):
    """Full field S (FP64, shape nz*ny*nx) of the same sum by zero-padded FFT.

    Builds the masked source ``I_h`` on the grid and the kernel table
    ``Gtab[d] = G(h |d|)`` for integer offsets d (``Gtab[0]`` = self term / h^3),
    then returns their linear (non-circular) convolution.  Values are exact up to
    FFT rounding (~1e-13 of the field's maximum), so this is a reference for
    rel-L2 over large target sets, not for small far-field values.
    """
    import scipy.fft as sfft
    vol = h ** 3
    src = np.zeros(nx * ny * nz, np.float64)
    J = np.asarray(J, np.int64)
    src[J] = source_scale * np.asarray(q, np.float64)[J] * vol
    src = src.reshape(nz, ny, nx)
    dz = np.arange(-(nz - 1), nz)
    dy = np.arange(-(ny - 1), ny)
    dx = np.arange(-(nx - 1), nx)
    DZ, DY, DX = np.meshgrid(dz, dy, dx, indexing="ij")
    R = h * np.sqrt((DX * DX + DY * DY + DZ * DZ).astype(np.float64))
    L = np.log(beta / alpha)
    with np.errstate(divide="ignore", invalid="ignore"):
        Gt = np.exp(-alpha * R) * (-np.expm1(-(beta - alpha) * R)) / (4 * np.pi * L * R ** 3)
    Gt[nz - 1, ny - 1, nx - 1] = self_integral(h, alpha, beta) / vol if self_mode == 1 else 0.0
    shape = (2 * nz - 1 + nz - 1, 2 * ny - 1 + ny - 1, 2 * nx - 1 + nx - 1)
    fshape = [sfft.next_fast_len(s) for s in shape]
    F = sfft.rfftn(src, fshape, workers=-1) * sfft.rfftn(Gt, fshape, workers=-1)
    full = sfft.irfftn(F, fshape, workers=-1)
    out = full[nz - 1:2 * nz - 1, ny - 1:2 * ny - 1, nx - 1:2 * nx - 1]
    return np.ascontiguousarray(out).ravel()


# ----------------------------------------------------------------------------
# Continuum reference for a spherically symmetric source (Eq. integral)
# ----------------------------------------------------------------------------

def radial_reference(r, I_of_rho, alpha, beta, rho_max):
    """S(r) of Eq. integral for a spherically symmetric emission I(rho).

    Integrating Eq. integral over the angles of y about the source centre gives
      S(r) = int_0^inf I(rho) rho/(2r) [F(r+rho) - F(|r-rho|)] drho,
      F(R) = [-e^{-alpha R}/R + alpha E1(alpha R) + e^{-beta R}/R - beta E1(beta R)] / L,
    an antiderivative of R*g(R)/R^2 * 4pi/(4pi) (d F/dR = (e^{-aR}-e^{-bR})/(L R^2)).
    F(|r-rho|) has a log singularity at rho = r, so the integral is split there.
    """
    import scipy.integrate as si
    import scipy.special as ss
    L = np.log(beta / alpha)

    def F(R):
        return (-np.exp(-alpha * R) / R + alpha * ss.exp1(alpha * R)
                + np.exp(-beta * R) / R - beta * ss.exp1(beta * R)) / L

    def f(rho):
        if rho == 0.0:
            return 0.0
        return I_of_rho(rho) * rho / (2 * r) * (F(r + rho) - F(abs(r - rho)))

    pts = [0.0, r, rho_max] if r < rho_max else [0.0, rho_max]
    tot = 0.0
    for a, b in zip(pts[:-1], pts[1:]):
        v, _ = si.quad(f, a, b, epsabs=0.0, epsrel=1e-13, limit=400)
        tot += v
    return tot


# ----------------------------------------------------------------------------
# Octree and interaction lists (plain recursive split + brute-force definitions)
# ----------------------------------------------------------------------------

def _coords(idx, nx, ny):
    idx = np.asarray(idx, np.int64)
    return idx % nx, (idx // nx) % ny, idx // (nx * ny)


def _morton(i, j, k, depth):
    key = np.zeros(np.shape(i), np.int64)
    for b in range(depth):
        key |= ((np.asarray(i, np.int64) >> b) & 1) << (3 * b)
        key |= ((np.asarray(j, np.int64) >> b) & 1) << (3 * b + 1)
        key |= ((np.asarray(k, np.int64) >> b) & 1) << (3 * b + 2)
    return key


def tree_depth(nx, ny, nz):
    """D: the grid is embedded at the origin corner of a 2^D cube of cells."""
    m = max(nx, ny, nz)
    D = 0
    while (1 << D) < m:
        D += 1
    return D


def octree(nx, ny, nz, J, T, leaf_size):
    """Octree over the selected sources J and targets T, plus U/V/W/X lists.

    Rules (an octree "such that each leaf cube contains no more than a
    prescribed number of points", Section 2.4):
      * the root is the 2^D cube of cells; a box exists if it holds any
        selected source or target;
      * a box at level l < D splits iff it holds more than ``leaf_size``
        sources or more than ``leaf_size`` targets; children are kept if
        non-empty;
      * Morton key interleaves x (bit 3b), y (3b+1), z (3b+2);
      * boxes are ordered by (level, key); points by Morton key.
    Lists, for boxes A (source side) and B (target side), with
    "adjacent" = the closed cubes touch or overlap:
      * U: B leaf with targets, A leaf with sources, A adjacent to B (near field, Eq. nearfar);
      * V: same level >= 2, B with targets, A with sources, parent(A) adjacent
        to parent(B), A not adjacent to B;
      * W: B leaf with targets, A with sources, level(A) > level(B),
        parent(A) adjacent to B, A not adjacent to B;
      * X: A leaf with sources, B with targets, level(B) > level(A),
        parent(B) adjacent to A, B not adjacent to A.
    Returns a dict of numpy arrays; list pairs are (target box, source box)
    indices sorted lexicographically.
    """
    D = tree_depth(nx, ny, nz)
    J = np.asarray(J, np.int64)
    T = np.asarray(T, np.int64)
    si, sj, sk = _coords(J, nx, ny)
    ti, tj, tk = _coords(T, nx, ny)
    skey = _morton(si, sj, sk, D)
    tkey = _morton(ti, tj, tk, D)
    sord = np.argsort(skey, kind="stable")
    tord = np.argsort(tkey, kind="stable")
    skey_s = skey[sord]
    tkey_s = tkey[tord]

    boxes = []   # (level, key, sb, se, tb, te, parent_index_in_list)

    def rec(level, key, sb, se, tb, te, parent):
        me = len(boxes)
        boxes.append([level, key, sb, se, tb, te, parent, 1])
        ns, nt = se - sb, te - tb
        if level < D and (ns > leaf_size or nt > leaf_size):
            boxes[me][7] = 0
            shift = 3 * (D - level - 1)
            for c in range(8):
                ck = key * 8 + c
                lo, hi = ck << shift, (ck + 1) << shift
                csb = sb + int(np.searchsorted(skey_s[sb:se], lo, "left"))
                cse = sb + int(np.searchsorted(skey_s[sb:se], hi, "left"))
                ctb = tb + int(np.searchsorted(tkey_s[tb:te], lo, "left"))
                cte = tb + int(np.searchsorted(tkey_s[tb:te], hi, "left"))
                if cse > csb or cte > ctb:
                    rec(level + 1, ck, csb, cse, ctb, cte, me)

    if J.size + T.size > 0:
        rec(0, 0, 0, J.size, 0, T.size, -1)
    B = np.array(boxes, dtype=np.int64).reshape(-1, 8)
    order = np.lexsort((B[:, 1], B[:, 0]))       # by level, then key
    inv = np.empty_like(order)
    inv[order] = np.arange(order.size)
    B = B[order]
    parent = np.where(B[:, 6] >= 0, inv[np.maximum(B[:, 6], 0)], -1)
    level, key = B[:, 0], B[:, 1]
    leaf = B[:, 7].astype(bool)
    ns = B[:, 3] - B[:, 2]
    nt = B[:, 5] - B[:, 4]

    # integer extents in cells: [lo, lo + size) per axis
    def decode(key, level):
        i = np.zeros_like(key)
        j = np.zeros_like(key)
        k = np.zeros_like(key)
        for b in range(D):
            i |= ((key >> (3 * b)) & 1) << b
            j |= ((key >> (3 * b + 1)) & 1) << b
            k |= ((key >> (3 * b + 2)) & 1) << b
        size = np.left_shift(1, D - level)
        return i * size, j * size, k * size, size

    bi, bj, bk, bs = decode(key, level)

    def adjacent(a, b):
        """closed cubes of boxes a and b (index arrays, broadcast) touch or overlap."""
        ok = np.ones(np.broadcast(a, b).shape, bool)
        for lo in (bi, bj, bk):
            ok &= (lo[a] <= lo[b] + bs[b]) & (lo[b] <= lo[a] + bs[a])
        return ok

    nb = len(B)
    idx = np.arange(nb)
    U, V, W, X = [], [], [], []
    for b in range(nb):                      # b: target-side box
        if nt[b] == 0:
            continue
        a = idx[ns > 0]
        adj = adjacent(a, np.full_like(a, b))
        if leaf[b]:
            sel = a[leaf[a] & adj]
            U += [(b, x) for x in sel]
            # W: finer boxes, parent adjacent to b, not adjacent to b
            cand = a[(level[a] > level[b]) & ~adj]
            if cand.size:
                padj = adjacent(parent[cand], np.full_like(cand, b))
                W += [(b, x) for x in cand[padj]]
        if level[b] >= 2:
            cand = a[(level[a] == level[b]) & ~adj]
            if cand.size:
                padj = adjacent(parent[cand], np.full_like(cand, parent[b]))
                V += [(b, x) for x in cand[padj]]
        if level[b] >= 1:
            cand = a[leaf[a] & (level[a] < level[b]) & ~adj]
            if cand.size:
                padj = adjacent(np.full_like(cand, parent[b]), cand)
                X += [(b, x) for x in cand[padj]]

    def pairs(lst):
        arr = np.array(lst, dtype=np.int64).reshape(-1, 2)
        if arr.size:
            arr = arr[np.lexsort((arr[:, 1], arr[:, 0]))]
        return arr

    return dict(depth=D, level=level, key=key, src_begin=B[:, 2], src_end=B[:, 3],
                trg_begin=B[:, 4], trg_end=B[:, 5], parent=parent, leaf=leaf,
                src_order=J[sord], trg_order=T[tord],
                U=pairs(U), V=pairs(V), W=pairs(W), X=pairs(X))
