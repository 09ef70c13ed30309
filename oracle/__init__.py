"""CPU oracle for the p-median GA of arXiv:1610.10061 -- test infrastructure.

Only the test-suite, ``__graft_entry__.smoke()`` and the benchmark's CPU
baseline may import this package.  The product library never does, and this
package never imports the product library.

Evaluators (three independent routes to the same number):

* ``eval_direct`` (O1) -- Section 1, Eqs. 1-3: sum over clients of the nearest
  open facility, straight from the distance matrix.
* ``hbp_polynomial`` / ``hbp_eval`` (O2) -- Section 2.1, Eq. 6 and Example 1:
  the Hammer-Beresnev polynomial over Pi'/Delta' as a dictionary of monomials
  in z = 1 - x, like monomials merged and zero coefficients dropped.
* ``eval_scan`` (O3) -- Section 4.2, the paper's Fitness function.

Plus ``tables`` (Section 2.1, Eq. 4 and truncation), ``cumulative`` /
``eval_cumulative`` (the running sums of Delta' read at the first open rank),
Philox4x32-10, Floyd sampling, the crossover (Section 4.3), shift mutation
(Section 4.4), the whole GA (Sections 3.1, 3.2.2, 4.5; Floyd or the
combinadic generation of Section 4.1 from ``combinadic.py``; migration
variants (i) and (ii)) and the swap statistics of the learned proposal
(``mlp.py`` holds its features, perceptron and Adam).  The C part lives in
``pm_oracle.c`` and is compiled with gcc into ``liboracle.so`` beside it on
first use.  ``ga_run``: parity unpinned by the paper (its Figures 1-3 are
missing); pinned by invariants, hand-worked operator cases and brute force.
"""

from __future__ import annotations

import ctypes
import itertools
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pm_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

OP_INIT = 0x001
OP_XOVER = 0x100
OP_MUT = 0x200


def build(force: bool = False) -> str:
    """Compile pm_oracle.c into liboracle.so (plain gcc -O2, no SIMD flags)."""
    stale = (not os.path.exists(_LIB)) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC)
    if force or stale:
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB)
    P = ctypes.c_void_p
    I64 = ctypes.c_int64
    U32 = ctypes.c_uint32
    U64 = ctypes.c_uint64
    lib.oracle_tables.argtypes = [P, I64, I64, I64, P, P]
    lib.oracle_eval_direct.argtypes = [P, I64, I64, P, I64, I64, P]
    lib.oracle_eval_scan.argtypes = [P, P, I64, I64, P, I64, I64, P, P]
    lib.oracle_brute_force.argtypes = [P, I64, I64, I64, I64, I64, P, P]
    lib.oracle_philox4x32_10.argtypes = [P, P, P]
    lib.oracle_philox4x32_10.restype = None
    lib.oracle_draw.argtypes = [U64, U32, U32, U32, U32, U32]
    lib.oracle_draw.restype = U32
    lib.oracle_uniform.argtypes = [U32, U32]
    lib.oracle_uniform.restype = U32
    lib.oracle_floyd_from_values.argtypes = [I64, I64, P, P]
    lib.oracle_floyd_from_values.restype = None
    lib.oracle_crossover.argtypes = [P, P, I64, I64, I64, P]
    lib.oracle_shift.argtypes = [P, I64, I64, I64, I64, ctypes.c_int, P]
    lib.oracle_shift.restype = None
    lib.oracle_mutation_params.argtypes = [U64, U32, U32, U32, U32, I64, P, P, P, P]
    lib.oracle_mutation_params.restype = None
    lib.oracle_crossover_params.argtypes = [U64, U32, U32, U32, U32, I64, I64, P, P]
    lib.oracle_crossover_params.restype = None
    lib.oracle_swap_stats.argtypes = [P, P, I64, I64, I64, P, I64, I64, P, P, P, P]
    lib.oracle_ga_run.argtypes = [P, P, I64, I64, I64, U64, U32, I64, I64, ctypes.c_int32, ctypes.c_int32,
                                  I64, I64, P, P, P, P, P, P, P, P, ctypes.c_int32, _INIT_FN, _EXTRA_FN]
    _lib = lib
    return lib


_INIT_FN = ctypes.CFUNCTYPE(None, ctypes.c_uint32, ctypes.c_uint32, ctypes.POINTER(ctypes.c_uint32))
_EXTRA_FN = ctypes.CFUNCTYPE(ctypes.c_int64, ctypes.c_uint32, ctypes.POINTER(ctypes.c_uint32),
                             ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_ubyte))


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _check(rc, what):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with code {rc}")


def mask_words(m: int) -> int:
    return (int(m) + 31) // 32


def _masks_from_sets(sets, m: int) -> np.ndarray:
    out = np.zeros((len(sets), mask_words(m)), dtype=np.uint32)
    for t, s in enumerate(sets):
        for j in s:
            out[t, j >> 5] |= np.uint32(1) << np.uint32(j & 31)
    return out


# --------------------------------------------------------------------------
# Section 2.1: orderings and increments
# --------------------------------------------------------------------------

def tables(d: np.ndarray, p: int | None = None, full: bool = False):
    """(Pi', Delta') with L = m-p+1 columns, or the full (Pi, Delta) if full=True.

    Pi holds 0-based facility ids as uint16, Delta int32 increments.
    """
    d = np.ascontiguousarray(d, dtype=np.int32)
    n, m = d.shape
    L = m if full else m - int(p) + 1
    pi = np.zeros((n, L), dtype=np.uint16)
    de = np.zeros((n, L), dtype=np.int32)
    _check(_load().oracle_tables(_ptr(d), n, m, L, _ptr(pi), _ptr(de)), "tables")
    return pi, de


# --------------------------------------------------------------------------
# Evaluators
# --------------------------------------------------------------------------

def eval_direct(d: np.ndarray, masks: np.ndarray) -> np.ndarray:
    """O1: sum_i min_{j open} d_ij per bitset row (Section 1, Eqs. 1-3)."""
    d = np.ascontiguousarray(d, dtype=np.int32)
    masks = np.ascontiguousarray(masks, dtype=np.uint32)
    n, m = d.shape
    P, W = masks.shape
    out = np.zeros(P, dtype=np.int64)
    _check(_load().oracle_eval_direct(_ptr(d), n, m, _ptr(masks), W, P, _ptr(out)), "eval_direct")
    return out


def eval_scan(pi: np.ndarray, delta: np.ndarray, masks: np.ndarray, return_ksum: bool = False):
    """O3: the paper's Fitness function over Pi'/Delta' (Section 4.2)."""
    pi = np.ascontiguousarray(pi, dtype=np.uint16)
    delta = np.ascontiguousarray(delta, dtype=np.int32)
    masks = np.ascontiguousarray(masks, dtype=np.uint32)
    n, L = pi.shape
    P, W = masks.shape
    out = np.zeros(P, dtype=np.int64)
    ks = np.zeros(1, dtype=np.int64)
    _check(_load().oracle_eval_scan(_ptr(pi), _ptr(delta), n, L, _ptr(masks), W, P, _ptr(out), _ptr(ks)),
           "eval_scan")
    return (out, int(ks[0])) if return_ksum else out


def cumulative(delta: np.ndarray) -> np.ndarray:
    """D' = the running sums of Delta' along each row (Eq. 4): D'_i[k] = sum_{s <= k} Delta'_i[s]."""
    return np.cumsum(np.asarray(delta, dtype=np.int64), axis=1)


def eval_cumulative(pi: np.ndarray, dcum: np.ndarray, masks: np.ndarray) -> np.ndarray:
    """O3 over cumulative tables: per client, D' at the first rank whose facility is open (no summing)."""
    pi = np.asarray(pi)
    dcum = np.asarray(dcum, dtype=np.int64)
    masks = np.ascontiguousarray(masks, dtype=np.uint32)
    n, L = pi.shape
    out = np.zeros(masks.shape[0], dtype=np.int64)
    for t, row in enumerate(masks):
        open_ = ((row[pi.astype(np.int64) >> 5] >> (pi.astype(np.uint32) & 31)) & 1).astype(bool)  # n x L
        first = open_.argmax(axis=1)
        if not open_[np.arange(n), first].all():
            raise RuntimeError("a client has no open facility within the truncated row")
        out[t] = int(dcum[np.arange(n), first].sum())
    return out


def hbp_polynomial(pi: np.ndarray, delta: np.ndarray) -> dict:
    """O2: the Hammer-Beresnev polynomial of Eq. 6 over Pi'/Delta'.

    Client i contributes delta_ik times the monomial prod_{r<k} z_{pi_ir}
    (k = 1 is the constant term).  Like monomials are merged and zero
    coefficients dropped, as in Example 1.  Keys are frozensets of 0-based
    facility ids (the empty set is the constant).
    """
    poly: dict = {}
    n, L = pi.shape
    for i in range(n):
        for k in range(L):
            mono = frozenset(int(j) for j in pi[i, :k])
            poly[mono] = poly.get(mono, 0) + int(delta[i, k])
    return {mono: c for mono, c in poly.items() if c != 0}


def hbp_eval(poly: dict, open_set) -> int:
    """Value of the polynomial at z_j = 1 - x_j for the given open facilities."""
    open_set = set(int(j) for j in open_set)
    return sum(c for mono, c in poly.items() if not (mono & open_set))


def brute_force(d: np.ndarray, p: int):
    """Minimum of O1 over all C(m, p) open sets: (cost, sorted facility tuple)."""
    d = np.ascontiguousarray(d, dtype=np.int32)
    m = d.shape[1]
    combos = list(itertools.combinations(range(m), p))
    best = None
    for s in range(0, len(combos), 4096):
        part = combos[s:s + 4096]
        c = eval_direct(d, _masks_from_sets(part, m))
        k = int(np.argmin(c))
        if best is None or c[k] < best[0]:
            best = (int(c[k]), part[k])
    return best


def brute_force_c(d: np.ndarray, p: int, threads: int | None = None):
    """Minimum of the objective over all C(m, p) open sets by the C enumeration (oracle_brute_force): one task per
    smallest facility a (the subsets whose smallest element is a), run on host threads; the smallest (cost,
    subset) wins, so ties go to the lexicographically first subset.  Returns (cost, sorted facility tuple)."""
    from concurrent.futures import ThreadPoolExecutor

    lib = _load()
    d = np.ascontiguousarray(d, dtype=np.int32)
    n, m = d.shape
    if threads is None:
        threads = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)

    def one(a):
        cost = np.zeros(1, dtype=np.int64)
        best = np.zeros(p, dtype=np.int32)
        _check(lib.oracle_brute_force(_ptr(d), n, m, p, a, a + 1, _ptr(cost), _ptr(best)), "brute_force")
        return int(cost[0]), tuple(int(j) for j in best)

    with ThreadPoolExecutor(max(1, threads)) as ex:
        results = list(ex.map(one, range(m - p + 1)))
    return min(results)


# --------------------------------------------------------------------------
# Random numbers and GA operators
# --------------------------------------------------------------------------

def philox4x32_10(ctr, key):
    c = np.asarray(ctr, dtype=np.uint32).copy()
    k = np.asarray(key, dtype=np.uint32).copy()
    out = np.zeros(4, dtype=np.uint32)
    _load().oracle_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def draw(seed: int, gen: int, unit: int, op: int, slot: int, inst: int = 0) -> int:
    return int(_load().oracle_draw(seed, gen, unit, op, slot, inst))


def uniform(u: int, N: int) -> int:
    return int(_load().oracle_uniform(u, N))


def floyd_from_values(m: int, p: int, values) -> np.ndarray:
    v = np.ascontiguousarray(values, dtype=np.uint32)
    x = np.zeros(mask_words(m), dtype=np.uint32)
    _load().oracle_floyd_from_values(m, p, _ptr(v), _ptr(x))
    return x


def crossover(C, couple, m: int, r1: int, i: int):
    C = np.ascontiguousarray(C, dtype=np.uint32)
    couple = np.ascontiguousarray(couple, dtype=np.uint32)
    F = np.zeros(mask_words(m), dtype=np.uint32)
    ok = _load().oracle_crossover(_ptr(C), _ptr(couple), m, r1, i, _ptr(F))
    return (F if ok else None)


def shift(C, m: int, a: int, length: int, k: int, right: bool):
    C = np.ascontiguousarray(C, dtype=np.uint32)
    F = np.zeros(mask_words(m), dtype=np.uint32)
    _load().oracle_shift(_ptr(C), m, a, length, k, int(bool(right)), _ptr(F))
    return F


def mutation_params(seed, gen, unit, q, m, inst=0):
    vals = [np.zeros(1, dtype=np.int64) for _ in range(3)]
    right = np.zeros(1, dtype=np.int32)
    _load().oracle_mutation_params(seed, gen, unit, q, inst, m, _ptr(vals[0]), _ptr(vals[1]), _ptr(vals[2]),
                                   _ptr(right))
    return int(vals[0][0]), int(vals[1][0]), int(vals[2][0]), bool(right[0])


def crossover_params(seed, gen, pair, r, m, p, inst=0):
    r1 = np.zeros(1, dtype=np.int64)
    i = np.zeros(1, dtype=np.int64)
    _load().oracle_crossover_params(seed, gen, pair, r, inst, m, p, _ptr(r1), _ptr(i))
    return int(r1[0]), int(i[0])


class GAState:
    """Resumable state of the oracle GA between generations."""

    def __init__(self, m: int, P: int, D: int):
        W = mask_words(m)
        self.deme_best = np.zeros((P // D, W), dtype=np.uint32)
        self.deme_cost = np.zeros(P // D, dtype=np.int64)
        self.best = np.zeros(W, dtype=np.uint32)
        self.scalars = np.array([-1, 0, 0, 0], dtype=np.int64)  # best_cost, sat, evals, next gen

    @property
    def best_cost(self):
        return int(self.scalars[0])

    @property
    def evals(self):
        return int(self.scalars[2])

    @property
    def generation(self):
        return int(self.scalars[3])


def ga_run(pi, delta, m: int, p: int, seed: int, P: int, D: int | None = None, gens: int = 1,
           xover_rounds: int | None = None, mut_tries: int | None = None, saturation: int = 0,
           state: GAState | None = None, record: bool = False, inst: int = 0, team: bool = False,
           init: str = "floyd", extra_try=None):
    """Run the reference GA for `gens` generations (Sections 3.1, 3.2.2, 4.5).

    team=True selects migration variant (ii) of Section 4.5 (all deme bests into deme 0).
    init="combinadic" draws fresh chromosomes as Section 4.1 does (oracle.combinadic), else Floyd sampling.
    extra_try(gen, X, c, enhanced) -> evaluations: a try between the crossover and the mutation cycles (the
    learned swap proposal, not in the paper) on the population X (P x W, writable), its costs c and the
    mutation cycle's `enhanced` flags (see oracle.mlp.first_candidate_try).

    Returns (state, trace, pops, costs); pops/costs are per-generation copies
    of the population after mutation when record=True.
    """
    pi = np.ascontiguousarray(pi, dtype=np.uint16)
    delta = np.ascontiguousarray(delta, dtype=np.int32)
    n = pi.shape[0]
    D = min(P, 256) if D is None else D
    lg = int(D).bit_length() - 1
    xover_rounds = lg if xover_rounds is None else xover_rounds
    mut_tries = lg if mut_tries is None else mut_tries
    W = mask_words(m)
    st = state if state is not None else GAState(m, P, D)
    trace = np.zeros(max(gens, 1), dtype=np.int64)
    pops = np.zeros((gens, P, W), dtype=np.uint32) if record else None
    costs = np.zeros((gens, P), dtype=np.int64) if record else None
    ran = np.zeros(1, dtype=np.int64)
    if init == "combinadic":
        from . import combinadic

        def fresh(g, t, x):
            words = combinadic.chromosome(seed, g, t, m, p, inst)
            for w in range(W):
                x[w] = int(words[w])

        init_fn = _INIT_FN(fresh)
    elif init == "floyd":
        init_fn = _INIT_FN()
    else:
        raise ValueError("init is 'floyd' or 'combinadic'")
    if extra_try is not None:
        def extra(g, xp, cp, ep):
            X = np.ctypeslib.as_array(xp, shape=(P, W))
            c = np.ctypeslib.as_array(cp, shape=(P,))
            e = np.ctypeslib.as_array(ep, shape=(P,))
            return int(extra_try(int(g), X, c, e))

        extra_fn = _EXTRA_FN(extra)
    else:
        extra_fn = _EXTRA_FN()
    rc = _load().oracle_ga_run(_ptr(pi), _ptr(delta), n, m, p, seed, inst, P, D, xover_rounds, mut_tries, gens,
                               saturation, _ptr(st.deme_best), _ptr(st.deme_cost), _ptr(st.best), _ptr(st.scalars),
                               _ptr(pops), _ptr(costs), _ptr(trace), _ptr(ran), 1 if team else 0, init_fn, extra_fn)
    _check(rc, "ga_run")
    k = int(ran[0])
    trace = trace[:k]
    if record:
        pops, costs = pops[:k], costs[:k]
    return st, trace, pops, costs


# --------------------------------------------------------------------------
# Swap statistics and move features (the learned swap proposal; not in the paper)
# --------------------------------------------------------------------------

def swap_stats(pi, delta, m: int, masks):
    """(gain, cap, loss, assign), each (P, m): see oracle_swap_stats in pm_oracle.c."""
    pi = np.ascontiguousarray(pi, dtype=np.uint16)
    delta = np.ascontiguousarray(delta, dtype=np.int32)
    masks = np.ascontiguousarray(masks, dtype=np.uint32)
    n, L = pi.shape
    P, W = masks.shape
    gain = np.zeros((P, m), dtype=np.int64)
    cap = np.zeros((P, m), dtype=np.int32)
    loss = np.zeros((P, m), dtype=np.int64)
    assign = np.zeros((P, m), dtype=np.int32)
    _check(_load().oracle_swap_stats(_ptr(pi), _ptr(delta), n, L, m, _ptr(masks), W, P, _ptr(gain), _ptr(cap),
                                     _ptr(loss), _ptr(assign)), "swap_stats")
    return gain, cap, loss, assign
