"""Thin ctypes binding of libpmgpu (include/pm.h), same names as the C ABI.

Only argument marshalling happens here; every step of the computation runs in
the library's CUDA kernels.  Arrays may be numpy arrays (host memory) or torch
CUDA tensors (device memory, used in place); torch supplies the stream
(``torch.cuda.current_stream()``) when it is available.

If ``libpmgpu.so`` is missing this module raises at import: there is no CPU
fallback.
"""

from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libpmgpu.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is not built; run `python -m paper_1610_10061_gb300.build` "
                      "(or __graft_entry__.build()) on a machine with nvcc")

_lib = ctypes.CDLL(LIB_PATH)

PM_OK = 0
STATUS = {0: "PM_OK", 1: "PM_ERR_INVALID_ARG", 2: "PM_ERR_NEGATIVE_DIST", 3: "PM_ERR_UNSUPPORTED",
          4: "PM_ERR_MASK", 5: "PM_ERR_CUDA", 6: "PM_ERR_OOM", 7: "PM_ERR_TIMEOUT"}


class PMError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = int(status)
        super().__init__(f"{where}: {pm_strerror(status)}")


class pm_ga_params(ctypes.Structure):
    _fields_ = [("deme", ctypes.c_int64), ("xover_rounds", ctypes.c_int32), ("mut_tries", ctypes.c_int32),
                ("saturation", ctypes.c_int64), ("stream_id", ctypes.c_uint32), ("flags", ctypes.c_uint32),
                ("model", ctypes.c_void_p), ("candidates", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class pm_eval_shape(ctypes.Structure):
    _fields_ = [("groups", ctypes.c_int32), ("warps", ctypes.c_int32), ("splits", ctypes.c_int32),
                ("grid", ctypes.c_int32), ("ms", ctypes.c_double), ("candidates", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


PM_GA_TUNE = 1
PM_TABLES_CUMULATIVE = 1
PM_GA_MIGRATE_TEAM = 2
PM_GA_INIT_COMBINADIC = 4


_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_PP = ctypes.POINTER(ctypes.c_void_p)
_S = ctypes.c_int

_SIGS = {
    "pm_strerror": ([_S], ctypes.c_char_p),
    "pm_instance_create": ([_P, _I64, _I64, _I64, ctypes.c_int, _P, _PP], _S),
    "pm_instance_create_ex": ([_P, _I64, _I64, _I64, ctypes.c_int, _P, ctypes.c_uint32, _PP], _S),
    "pm_instance_flags": ([_P, ctypes.POINTER(ctypes.c_uint32)], _S),
    "pm_instance_destroy": ([_P], _S),
    "pm_instance_info": ([_P, _P, _P, _P, _P, _P, _P], _S),
    "pm_instance_tables": ([_P, _P, _P, _P], _S),
    "pm_eval_population": ([_P, _P, _I64, _P, ctypes.c_int, _P], _S),
    "pm_eval_population_noalloc": ([_P, _P, _I64, _P, _P], _S),
    "pm_selftest_bounded_wait": ([ctypes.c_int, _P], _S),
    "pm_debug_fail_alloc": ([_I64, _P], _S),
    "pm_debug_scan_timeout": ([_I64, _P], _S),
    "pm_eval_status": ([_P, _P], _S),
    "pm_columns_layout": ([_P, _I64, _P, _P], _S),
    "pm_population_columns": ([_P, _P, _I64, _P, _P], _S),
    "pm_eval_columns": ([_P, _P, _I64, _P, _P], _S),
    "pm_tune_eval": ([_P, _I64, _P, ctypes.POINTER(pm_eval_shape)], _S),
    "pm_set_eval_shape": ([_P, _I64, ctypes.POINTER(pm_eval_shape)], _S),
    "pm_ga_create": ([_P, ctypes.c_uint64, _I64, ctypes.POINTER(pm_ga_params), _P, _PP], _S),
    "pm_ga_step": ([_P, _I64, _P, _P], _S),
    "pm_ga_result": ([_P, _P, _P, _P, _P, _P], _S),
    "pm_ga_population": ([_P, _P, _P, _P], _S),
    "pm_ga_save": ([_P, _P, ctypes.POINTER(ctypes.c_size_t), _P], _S),
    "pm_ga_load": ([_P, _P, ctypes.c_size_t, _P, _PP], _S),
    "pm_ga_destroy": ([_P], _S),
    "pm_ga_info": ([_P, _P, _P, _P, _P, _P, _P], _S),
    "pm_ga_instance_result": ([_P, _I64, _P, _P, _P, _P, _P], _S),
    "pm_ga_instance_population": ([_P, _I64, _P, _P, _P], _S),
    "pm_batch_create": ([_P, _I64, _PP], _S),
    "pm_batch_destroy": ([_P], _S),
    "pm_batch_eval": ([_P, _P, _P, _P, _P], _S),
    "pm_batch_tune": ([_P, _P, _P, ctypes.POINTER(pm_eval_shape)], _S),
    "pm_batch_ga_create": ([_P, ctypes.c_uint64, _I64, ctypes.POINTER(pm_ga_params), _P, _PP], _S),
    "pm_model_num_params": ([], ctypes.c_int64),
    "pm_model_create": ([ctypes.c_int, ctypes.c_uint64, _PP], _S),
    "pm_model_destroy": ([_P], _S),
    "pm_model_set_params": ([_P, _P, _P], _S),
    "pm_model_get_params": ([_P, _P, _P], _S),
    "pm_model_forward": ([_P, _P, _I64, _P, _P], _S),
    "pm_model_grad": ([_P, _P, _P, _I64, _P, _P, _P], _S),
    "pm_model_train_step": ([_P, _P, _P, _I64, ctypes.c_float, _P, _P], _S),
    "pm_hbp_create": ([_P, _P, _P], _S),
    "pm_hbp_destroy": ([_P], _S),
    "pm_hbp_info": ([_P, _P, _P], _S),
    "pm_hbp_terms": ([_P, _P, _P, _P], _S),
    "pm_hbp_eval": ([_P, _P, _I64, _P, _P], _S),
    "pm_model_train": ([_P, _P, _P, _I64, ctypes.c_int32, _I64, ctypes.c_float, ctypes.c_uint64, _P, _P], _S),
    "pm_swap_stats": ([_P, _P, _I64, _P, _P, _P, _P, _P], _S),
    "pm_move_features": ([_P, _P, _P, _P, _P, _P, _P, _I64, _I64, _P, _P], _S),
    "pm_log_moves": ([_P, _P, _P, _I64, _I64, ctypes.c_uint64, _P, _P, _P, _P], _S),
    "pm_ga_run": ([_P, ctypes.c_uint64, _I64, _I64, ctypes.POINTER(pm_ga_params), _P, _P, _P, _P, _P, _P], _S),
}
for _name, (_args, _res) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = _res


def exported_symbols():
    """Names this binding expects the library to export."""
    return sorted(_SIGS)


def pm_strerror(status: int) -> str:
    return _lib.pm_strerror(int(status)).decode()


def _check(status: int, where: str):
    if status != PM_OK:
        raise PMError(status, where)


def _stream(stream):
    if stream is not None:
        return ctypes.c_void_p(int(stream))
    try:
        import torch
        if torch.cuda.is_available() and torch.cuda.is_initialized():
            return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    except Exception:
        pass
    return ctypes.c_void_p(0)


def _addr(a):
    """Address of a numpy array or a torch tensor (CPU or CUDA); None -> NULL."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return ctypes.c_void_p(a.ctypes.data)
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(a.data_ptr())
    raise TypeError(f"unsupported buffer type {type(a)}")


# --------------------------------------------------------------------------
# Same-name wrappers of the C ABI (marshalling only)
# --------------------------------------------------------------------------

def pm_instance_create(d, n: int, m: int, p: int, device: int = 0, stream=None):
    out = ctypes.c_void_p()
    _check(_lib.pm_instance_create(_addr(d), n, m, p, device, _stream(stream), ctypes.byref(out)),
           "pm_instance_create")
    return out


def pm_instance_create_ex(d, n: int, m: int, p: int, device: int = 0, stream=None, flags: int = 0):
    out = ctypes.c_void_p()
    _check(_lib.pm_instance_create_ex(_addr(d), n, m, p, device, _stream(stream), flags, ctypes.byref(out)),
           "pm_instance_create_ex")
    return out


def pm_instance_flags(inst) -> int:
    out = ctypes.c_uint32()
    _check(_lib.pm_instance_flags(inst, ctypes.byref(out)), "pm_instance_flags")
    return int(out.value)


def pm_instance_destroy(inst):
    _check(_lib.pm_instance_destroy(inst), "pm_instance_destroy")


def pm_instance_info(inst):
    vals = [ctypes.c_int64() for _ in range(6)]
    _check(_lib.pm_instance_info(inst, *[ctypes.byref(v) for v in vals]), "pm_instance_info")
    return dict(zip(["n", "m", "p", "L", "W", "stride"], [v.value for v in vals]))


def pm_instance_tables(inst, pi_out, delta_out, stream=None):
    _check(_lib.pm_instance_tables(inst, _addr(pi_out), _addr(delta_out), _stream(stream)), "pm_instance_tables")


def pm_eval_population(inst, masks, pop: int, costs, checked: int = 0, stream=None):
    _check(_lib.pm_eval_population(inst, _addr(masks), pop, _addr(costs), int(checked), _stream(stream)),
           "pm_eval_population")


def pm_eval_population_noalloc(inst, masks, pop: int, costs, stream=None):
    _check(_lib.pm_eval_population_noalloc(inst, _addr(masks), pop, _addr(costs), _stream(stream)),
           "pm_eval_population_noalloc")


def pm_selftest_bounded_wait(device: int = 0, stream=None) -> int:
    """Status recorded by a kernel whose wait can never complete (PM_ERR_TIMEOUT = 7 when the bound works)."""
    return int(_lib.pm_selftest_bounded_wait(device, _stream(stream)))


def pm_debug_fail_alloc(after: int) -> int:
    """Make the library's device allocation after `after` more successful ones fail with PM_ERR_OOM (negative:
    off).  Returns the allocations that were still to succeed before the previously armed failure (-1: none armed,
    or it has happened)."""
    pending = ctypes.c_int64(-1)
    _check(_lib.pm_debug_fail_alloc(int(after), ctypes.byref(pending)), "pm_debug_fail_alloc")
    return int(pending.value)


def pm_debug_scan_timeout(launches: int) -> int:
    """Arm the next `launches` column-scan launches to skip their tile copy, so that their bounded wait runs out
    (PM_ERR_TIMEOUT, no fault).  Returns the launches that were still armed."""
    pending = ctypes.c_int64(0)
    _check(_lib.pm_debug_scan_timeout(int(launches), ctypes.byref(pending)), "pm_debug_scan_timeout")
    return int(pending.value)


def pm_eval_status(inst, stream=None) -> int:
    """Status of the asynchronous evaluations on inst since the last report (0 or PM_ERR_TIMEOUT = 7); clears
    the record."""
    return int(_lib.pm_eval_status(inst, _stream(stream)))


def pm_columns_layout(inst, pop: int):
    """(G, words) of the facility-major form the evaluation of `pop` individuals uses."""
    g = ctypes.c_int32()
    w = ctypes.c_int64()
    _check(_lib.pm_columns_layout(inst, pop, ctypes.byref(g), ctypes.byref(w)), "pm_columns_layout")
    return int(g.value), int(w.value)


def pm_population_columns(inst, masks, pop: int, cols, stream=None):
    _check(_lib.pm_population_columns(inst, _addr(masks), pop, _addr(cols), _stream(stream)), "pm_population_columns")


def pm_eval_columns(inst, cols, pop: int, costs, stream=None):
    _check(_lib.pm_eval_columns(inst, _addr(cols), pop, _addr(costs), _stream(stream)), "pm_eval_columns")


def pm_tune_eval(inst, pop: int, stream=None):
    out = pm_eval_shape()
    _check(_lib.pm_tune_eval(inst, pop, _stream(stream), ctypes.byref(out)), "pm_tune_eval")
    return dict(groups=out.groups, warps=out.warps, splits=out.splits, grid=out.grid, ms=out.ms,
                candidates=out.candidates)


def pm_set_eval_shape(inst, pop: int, groups: int, warps: int = 16, splits: int = 0):
    shape = pm_eval_shape(groups, warps, splits, 0, 0.0, 0, 0)
    _check(_lib.pm_set_eval_shape(inst, pop, ctypes.byref(shape)), "pm_set_eval_shape")


def _params(deme=0, xover_rounds=-1, mut_tries=-1, saturation=0, stream_id=0, tune=False, model=None,
            candidates=0, migration="deme", init="floyd"):
    if migration not in ("deme", "team"):
        raise ValueError("migration is 'deme' (variant (i)) or 'team' (variant (ii))")
    if init not in ("floyd", "combinadic"):
        raise ValueError("init is 'floyd' or 'combinadic'")
    mh = model.handle if isinstance(model, Model) else model
    flags = ((PM_GA_TUNE if tune else 0) | (PM_GA_MIGRATE_TEAM if migration == "team" else 0)
             | (PM_GA_INIT_COMBINADIC if init == "combinadic" else 0))
    return pm_ga_params(deme, xover_rounds, mut_tries, saturation, stream_id, flags,
                        mh if mh is not None else None, candidates, 0)


# ----- learned swap proposal -----

def pm_model_num_params() -> int:
    return int(_lib.pm_model_num_params())


def pm_model_create(device: int = 0, seed: int = 0):
    out = ctypes.c_void_p()
    _check(_lib.pm_model_create(device, seed, ctypes.byref(out)), "pm_model_create")
    return out


def pm_model_destroy(md):
    _check(_lib.pm_model_destroy(md), "pm_model_destroy")


def pm_model_set_params(md, params, stream=None):
    _check(_lib.pm_model_set_params(md, _addr(params), _stream(stream)), "pm_model_set_params")


def pm_model_get_params(md, params, stream=None):
    _check(_lib.pm_model_get_params(md, _addr(params), _stream(stream)), "pm_model_get_params")


def pm_model_forward(md, x, rows: int, y, stream=None):
    _check(_lib.pm_model_forward(md, _addr(x), rows, _addr(y), _stream(stream)), "pm_model_forward")


def pm_model_grad(md, x, t, rows: int, grads=None, stream=None) -> float:
    loss = ctypes.c_float()
    _check(_lib.pm_model_grad(md, _addr(x), _addr(t), rows, _addr(grads), ctypes.byref(loss), _stream(stream)),
           "pm_model_grad")
    return loss.value


def pm_model_train_step(md, x, t, rows: int, lr: float, want_loss: bool = False, stream=None):
    loss = ctypes.c_float()
    _check(_lib.pm_model_train_step(md, _addr(x), _addr(t), rows, lr, ctypes.byref(loss) if want_loss else None,
                                    _stream(stream)), "pm_model_train_step")
    return loss.value if want_loss else None


def pm_hbp_create(inst, stream=None):
    h = ctypes.c_void_p()
    _check(_lib.pm_hbp_create(inst, _stream(stream), ctypes.byref(h)), "pm_hbp_create")
    return h


def pm_hbp_destroy(h):
    _check(_lib.pm_hbp_destroy(h), "pm_hbp_destroy")


def pm_hbp_info(h):
    terms, W = ctypes.c_int64(), ctypes.c_int64()
    _check(_lib.pm_hbp_info(h, ctypes.byref(terms), ctypes.byref(W)), "pm_hbp_info")
    return int(terms.value), int(W.value)


def pm_hbp_terms(h, sets, coeffs, stream=None):
    _check(_lib.pm_hbp_terms(h, _addr(sets), _addr(coeffs), _stream(stream)), "pm_hbp_terms")


def pm_hbp_eval(h, masks, pop: int, costs, stream=None):
    _check(_lib.pm_hbp_eval(h, _addr(masks), int(pop), _addr(costs), _stream(stream)), "pm_hbp_eval")


class Polynomial:
    """The reduced Hammer-Beresnev polynomial of an Instance, built and evaluated on the device."""

    def __init__(self, inst, stream=None):
        self.inst = inst
        self.handle = pm_hbp_create(inst.handle, stream)
        self.terms, self.W = pm_hbp_info(self.handle)

    def monomials(self):
        """{frozenset of facility ids: coefficient} (host)."""
        sets = np.zeros((max(self.terms, 1), self.W), dtype=np.uint32)
        coeffs = np.zeros(max(self.terms, 1), dtype=np.int64)
        pm_hbp_terms(self.handle, sets, coeffs)
        out = {}
        for q in range(self.terms):
            bits = np.nonzero(np.unpackbits(sets[q].view(np.uint8), bitorder="little"))[0]
            out[frozenset(int(j) for j in bits)] = int(coeffs[q])
        return out

    def eval(self, masks, costs=None, stream=None):
        """Values at a device population (torch CUDA tensor of pop x W int32 words)."""
        import torch

        pop = int(masks.shape[0])
        if costs is None:
            costs = torch.empty(pop, dtype=torch.int64, device=masks.device)
        pm_hbp_eval(self.handle, masks, pop, costs, stream)
        return costs

    def close(self):
        if self.handle:
            pm_hbp_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pm_model_train(model, x, t, rows: int, epochs: int, batch: int, lr: float, seed: int, losses=None, stream=None):
    _check(_lib.pm_model_train(model, _addr(x), _addr(t), int(rows), int(epochs), int(batch), ctypes.c_float(lr),
                               ctypes.c_uint64(seed), _addr(losses), _stream(stream)), "pm_model_train")


def pm_swap_stats(inst, masks, pop: int, gain, cap, loss, assign, stream=None):
    _check(_lib.pm_swap_stats(inst, _addr(masks), pop, _addr(gain), _addr(cap), _addr(loss), _addr(assign),
                              _stream(stream)), "pm_swap_stats")


def pm_move_features(inst, gain, cap, loss, assign, costs, moves, pop: int, C: int, x, stream=None):
    _check(_lib.pm_move_features(inst, _addr(gain), _addr(cap), _addr(loss), _addr(assign), _addr(costs),
                                 _addr(moves), pop, C, _addr(x), _stream(stream)), "pm_move_features")


def pm_log_moves(inst, masks, costs, pop: int, per: int, seed: int, x, t, moves, stream=None):
    _check(_lib.pm_log_moves(inst, _addr(masks), _addr(costs), pop, per, seed, _addr(x), _addr(t), _addr(moves),
                             _stream(stream)), "pm_log_moves")


class Model:
    """The swap-scoring perceptron (16 -> 128 -> 128 -> 1) on the device."""

    def __init__(self, device: int = 0, seed: int = 0):
        self.handle = pm_model_create(device, seed)
        self.n_params = pm_model_num_params()

    def params(self):
        out = np.zeros(self.n_params, dtype=np.float32)
        pm_model_get_params(self.handle, out)
        return out

    def set_params(self, params):
        pm_model_set_params(self.handle, np.ascontiguousarray(params, dtype=np.float32))

    def forward(self, x, stream=None):
        import torch
        y = torch.empty(x.shape[0], dtype=torch.float32, device=x.device)
        pm_model_forward(self.handle, x, x.shape[0], y, stream)
        return y

    def grad(self, x, t):
        g = np.zeros(self.n_params, dtype=np.float32)
        loss = pm_model_grad(self.handle, x, t, x.shape[0], g)
        return loss, g

    def train(self, x, t, epochs: int = 3, batch: int = 4096, lr: float = 1e-3, seed: int = 0, stream=None):
        """Adam on (x, t) (device tensors) in mini-batches shuffled on the device (pm_model_train); returns the
        loss of every step (numpy, float32)."""
        rows = int(x.shape[0])
        steps = int(epochs) * (-(-rows // int(batch)))
        losses = np.zeros(max(steps, 1), dtype=np.float32)
        pm_model_train(self.handle, x, t, rows, int(epochs), int(batch), float(lr), int(seed), losses, stream)
        return losses[:steps]

    def close(self):
        if self.handle:
            pm_model_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pm_ga_create(inst, seed: int, pop: int, params: pm_ga_params | None = None, stream=None):
    out = ctypes.c_void_p()
    _check(_lib.pm_ga_create(inst, seed, pop, ctypes.byref(params) if params is not None else None,
                             _stream(stream), ctypes.byref(out)), "pm_ga_create")
    return out


def pm_ga_step(ga, gens: int, trace=None, stream=None):
    _check(_lib.pm_ga_step(ga, gens, _addr(trace), _stream(stream)), "pm_ga_step")


def pm_ga_result(ga, best_mask=None, stream=None):
    bc, gr, ev = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    _check(_lib.pm_ga_result(ga, ctypes.byref(bc), _addr(best_mask), ctypes.byref(gr), ctypes.byref(ev),
                             _stream(stream)), "pm_ga_result")
    return bc.value, gr.value, ev.value


def pm_ga_population(ga, masks, costs, stream=None):
    _check(_lib.pm_ga_population(ga, _addr(masks), _addr(costs), _stream(stream)), "pm_ga_population")


def pm_ga_save(ga, stream=None) -> bytes:
    n = ctypes.c_size_t(0)
    _check(_lib.pm_ga_save(ga, None, ctypes.byref(n), _stream(stream)), "pm_ga_save")
    buf = ctypes.create_string_buffer(n.value)
    _check(_lib.pm_ga_save(ga, buf, ctypes.byref(n), _stream(stream)), "pm_ga_save")
    return buf.raw[: n.value]


def pm_ga_load(inst, blob: bytes, stream=None):
    out = ctypes.c_void_p()
    buf = ctypes.create_string_buffer(blob, len(blob))
    _check(_lib.pm_ga_load(inst, buf, len(blob), _stream(stream), ctypes.byref(out)), "pm_ga_load")
    return out


def pm_ga_info(ga):
    pop, deme, kg, ks = (ctypes.c_int64() for _ in range(4))
    xr, mt = ctypes.c_int32(), ctypes.c_int32()
    _check(_lib.pm_ga_info(ga, ctypes.byref(pop), ctypes.byref(deme), ctypes.byref(xr), ctypes.byref(mt),
                           ctypes.byref(kg), ctypes.byref(ks)), "pm_ga_info")
    return dict(pop=pop.value, deme=deme.value, xover_rounds=xr.value, mut_tries=mt.value,
                kernels_per_generation=kg.value, kernels_per_step_call=ks.value)


def pm_ga_instance_result(ga, k: int, best_mask=None, stream=None):
    bc, gr, ev = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    _check(_lib.pm_ga_instance_result(ga, k, ctypes.byref(bc), _addr(best_mask), ctypes.byref(gr), ctypes.byref(ev),
                                      _stream(stream)), "pm_ga_instance_result")
    return bc.value, gr.value, ev.value


def pm_ga_instance_population(ga, k: int, masks, costs, stream=None):
    _check(_lib.pm_ga_instance_population(ga, k, _addr(masks), _addr(costs), _stream(stream)),
           "pm_ga_instance_population")


def pm_batch_create(inst_handles):
    arr = (ctypes.c_void_p * len(inst_handles))(*[h.value for h in inst_handles])
    out = ctypes.c_void_p()
    _check(_lib.pm_batch_create(arr, len(inst_handles), ctypes.byref(out)), "pm_batch_create")
    return out


def pm_batch_destroy(b):
    _check(_lib.pm_batch_destroy(b), "pm_batch_destroy")


def pm_batch_eval(b, masks, pops, costs, stream=None):
    pv = np.ascontiguousarray(pops, dtype=np.int64)
    _check(_lib.pm_batch_eval(b, _addr(masks), _addr(pv), _addr(costs), _stream(stream)), "pm_batch_eval")


def pm_batch_tune(b, pops, stream=None):
    pv = np.ascontiguousarray(pops, dtype=np.int64)
    out = pm_eval_shape()
    _check(_lib.pm_batch_tune(b, _addr(pv), _stream(stream), ctypes.byref(out)), "pm_batch_tune")
    return dict(groups=out.groups, warps=out.warps, items_per_cta=out.splits, grid=out.grid, ms=out.ms,
                candidates=out.candidates)


def pm_batch_ga_create(b, seed: int, pop: int, params: pm_ga_params | None = None, stream=None):
    out = ctypes.c_void_p()
    _check(_lib.pm_batch_ga_create(b, seed, pop, ctypes.byref(params) if params is not None else None,
                                   _stream(stream), ctypes.byref(out)), "pm_batch_ga_create")
    return out


def pm_ga_destroy(ga):
    _check(_lib.pm_ga_destroy(ga), "pm_ga_destroy")


def pm_ga_run(inst, seed: int, pop: int, gens: int, params: pm_ga_params | None = None, best_mask=None,
              trace=None, stream=None):
    bc, gr, ev = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    _check(_lib.pm_ga_run(inst, seed, pop, gens, ctypes.byref(params) if params is not None else None,
                          ctypes.byref(bc), _addr(best_mask), ctypes.byref(gr), ctypes.byref(ev), _addr(trace),
                          _stream(stream)), "pm_ga_run")
    return bc.value, gr.value, ev.value


# --------------------------------------------------------------------------
# Small object layer for Python callers
# --------------------------------------------------------------------------

class Instance:
    """A p-median instance with its device-resident Pi'/Delta' tables."""

    def __init__(self, d, p: int, device: int = 0, stream=None, cumulative: bool = False):
        """cumulative=True keeps D' (running sums of Delta') on the device (PM_TABLES_CUMULATIVE)."""
        if isinstance(d, np.ndarray):
            d = np.ascontiguousarray(d, dtype=np.int32)
        n, m = int(d.shape[0]), int(d.shape[1])
        if cumulative:
            self.handle = pm_instance_create_ex(d, n, m, int(p), device, stream, PM_TABLES_CUMULATIVE)
        else:
            self.handle = pm_instance_create(d, n, m, int(p), device, stream)
        self.cumulative = bool(cumulative)
        info = pm_instance_info(self.handle)
        self.n, self.m, self.p, self.L, self.W, self.stride = (info[k] for k in ("n", "m", "p", "L", "W", "stride"))

    def tables(self, stream=None):
        pi = np.zeros((self.n, self.L), dtype=np.uint16)
        de = np.zeros((self.n, self.L), dtype=np.int32)
        pm_instance_tables(self.handle, pi, de, stream)
        return pi, de

    def eval(self, masks, costs=None, checked: bool = False, stream=None):
        """Costs of a population; numpy in -> numpy out, CUDA tensor in -> CUDA tensor out."""
        pop = int(masks.shape[0]) if masks.ndim == 2 else int(masks.shape[0] // self.W)
        if costs is None:
            if isinstance(masks, np.ndarray):
                costs = np.zeros(pop, dtype=np.int64)
            else:
                import torch
                costs = torch.empty(pop, dtype=torch.int64, device=masks.device)
        pm_eval_population(self.handle, masks, pop, costs, int(checked), stream)
        return costs

    def tune(self, pop: int, stream=None):
        """Autotune the evaluation tile shape for populations of `pop` (see pm_tune_eval)."""
        return pm_tune_eval(self.handle, int(pop), stream)

    def set_shape(self, pop: int, groups: int, warps: int = 16, splits: int = 0):
        """Pin the evaluation tile shape for populations of `pop` (see pm_set_eval_shape)."""
        pm_set_eval_shape(self.handle, int(pop), groups, warps, splits)

    def close(self):
        if self.handle:
            pm_instance_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class GA:
    """The device-resident genetic algorithm on an Instance."""

    def __init__(self, inst: Instance, seed: int, pop: int, deme: int = 0, xover_rounds: int = -1,
                 mut_tries: int = -1, saturation: int = 0, stream_id: int = 0, tune: bool = False, model=None,
                 candidates: int = 0, migration: str = "deme", init: str = "floyd", stream=None, _handle=None):
        self.inst = inst
        self.pop = int(pop)
        self.model = model
        self.handle = _handle if _handle is not None else pm_ga_create(
            inst.handle, seed, pop,
            _params(deme, xover_rounds, mut_tries, saturation, stream_id, tune, model, candidates, migration, init),
            stream)

    def step(self, gens: int, stream=None):
        trace = np.zeros(max(int(gens), 1), dtype=np.int64)
        before = self.result(stream)[1]
        pm_ga_step(self.handle, int(gens), trace, stream)
        ran = self.result(stream)[1] - before
        return trace[:ran]

    def result(self, stream=None):
        mask = np.zeros(self.inst.W, dtype=np.uint32)
        bc, gr, ev = pm_ga_result(self.handle, mask, stream)
        return bc, gr, ev, mask

    def population(self, stream=None):
        masks = np.zeros((self.pop, self.inst.W), dtype=np.uint32)
        costs = np.zeros(self.pop, dtype=np.int64)
        pm_ga_population(self.handle, masks, costs, stream)
        return masks, costs

    def save(self, stream=None) -> bytes:
        return pm_ga_save(self.handle, stream)

    def info(self):
        return pm_ga_info(self.handle)

    @classmethod
    def load(cls, inst: Instance, blob: bytes, stream=None):
        h = pm_ga_load(inst.handle, blob, stream)
        return cls(inst, 0, pm_ga_info(h)["pop"], _handle=h)

    def close(self):
        if self.handle:
            pm_ga_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Several instances evaluated (and evolved) together in single launches."""

    def __init__(self, instances):
        self.instances = list(instances)
        self.handle = pm_batch_create([i.handle for i in self.instances])

    def eval(self, masks, pops, costs=None, stream=None):
        """masks: device tensor of the populations back to back; returns a device tensor of sum(pops) costs."""
        import torch

        if costs is None:
            costs = torch.empty(int(sum(pops)), dtype=torch.int64, device=masks.device)
        pm_batch_eval(self.handle, masks, pops, costs, stream)
        return costs

    def tune(self, pops, stream=None):
        return pm_batch_tune(self.handle, pops, stream)

    def ga(self, seed: int, pop: int, deme: int = 0, xover_rounds: int = -1, mut_tries: int = -1,
           saturation: int = 0, stream_id: int = 0, tune: bool = False, migration: str = "deme", stream=None):
        h = pm_batch_ga_create(self.handle, seed, pop,
                               _params(deme, xover_rounds, mut_tries, saturation, stream_id, tune,
                                       migration=migration), stream)
        return BatchGA(self, pop, h)

    def close(self):
        if self.handle:
            pm_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BatchGA:
    """A GA per instance of a Batch, stepped together."""

    def __init__(self, batch: Batch, pop: int, handle):
        self.batch = batch
        self.pop = int(pop)
        self.handle = handle
        self.K = len(batch.instances)

    def step(self, gens: int, stream=None):
        """Run `gens` generations; returns a (K, gens) trace (entries past an instance's stop are unspecified)."""
        trace = np.zeros((self.K, max(int(gens), 1)), dtype=np.int64)
        pm_ga_step(self.handle, int(gens), trace, stream)
        return trace[:, :int(gens)]

    def result(self, k: int, stream=None):
        mask = np.zeros(self.batch.instances[k].W, dtype=np.uint32)
        bc, gr, ev = pm_ga_instance_result(self.handle, k, mask, stream)
        return bc, gr, ev, mask

    def population(self, k: int, stream=None):
        W = self.batch.instances[k].W
        masks = np.zeros((self.pop, W), dtype=np.uint32)
        costs = np.zeros(self.pop, dtype=np.int64)
        pm_ga_instance_population(self.handle, k, masks, costs, stream)
        return masks, costs

    def info(self):
        return pm_ga_info(self.handle)

    def close(self):
        if self.handle:
            pm_ga_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
