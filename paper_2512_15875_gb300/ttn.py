"""Thin ctypes binding of ``libttn.so`` (the C ABI declared in ``include/ttn.h``).

Every function here has the name of the C entry point it wraps and only marshals arguments
(NumPy arrays <-> pointers, handles, status codes -> exceptions). All computation happens in the
library. There is no fallback: if the library is missing, every call raises.
"""
from __future__ import annotations

import atexit
import ctypes as C
import os
import weakref

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libttn.so")

TTN_FP64, TTN_FP32, TTN_TF32X3, TTN_TF32X3_TC05 = 0, 1, 2, 3
TTN_MAX_LEGS = 8
STATUS = {0: "TTN_OK", 1: "TTN_EINVAL", 2: "TTN_ENOMEM", 3: "TTN_ECUDA", 4: "TTN_ENONFINITE",
          5: "TTN_ENOTCONV", 6: "TTN_ETIMEOUT", 7: "TTN_EUNSUPPORTED"}
PRECISION = {"fp64": TTN_FP64, "fp32": TTN_FP32, "tf32x3": TTN_TF32X3,
             "tf32x3_tc05": TTN_TF32X3_TC05}

_lib = None
_P = C.c_void_p
_I = C.c_int
_LL = C.c_longlong
_D = C.c_double
_IP = C.POINTER(C.c_int)
_LLP = C.POINTER(C.c_longlong)
_DP = C.POINTER(C.c_double)

_SIGS = {
    "ttn_create": (_I, [C.POINTER(_P), _I, _P]),
    "ttn_destroy": (None, [_P]),
    "ttn_last_error": (C.c_char_p, [_P]),
    "ttn_synchronize": (_I, [_P]),
    "ttn_launch_count": (_LL, [_P]),
    "ttn_flop_count": (_D, [_P]),
    "ttn_profile_enable": (_I, [_P, _I]),
    "ttn_profile_get": (_I, [_P, _I, C.c_char_p, _LLP, _DP, _DP, _DP, _IP]),
    "ttn_tree_create": (_I, [_P, _I, _IP, _IP, C.POINTER(_P)]),
    "ttn_tree_destroy": (None, [_P]),
    "ttn_build_ttno": (_I, [_P, _P, _I, _IP, _LLP, _DP, _I, _DP, _IP, _IP, _D, C.POINTER(_P),
                            _IP]),
    "ttn_ttno_create": (_I, [_P, _P, _IP, _I, _IP, _LLP, _DP, _I, _IP, _IP, _IP, _DP,
                             C.POINTER(_P)]),
    "ttn_ttno_info": (_I, [_P, _IP, _IP, _LLP]),
    "ttn_ttno_get_entries": (_I, [_P, _IP, _IP, _DP, _LLP, _DP]),
    "ttn_ttno_destroy": (None, [_P]),
    "ttn_block_create": (_I, [_P, _P, _I, _IP, C.POINTER(_P)]),
    "ttn_block_destroy": (None, [_P]),
    "ttn_block_set": (_I, [_P, _I, _I, _DP, _LL]),
    "ttn_block_get": (_I, [_P, _I, _I, _DP, _LL]),
    "ttn_block_node_info": (_I, [_P, _I, _LLP, C.POINTER(_DP)]),
    "ttn_block_copy_states": (_I, [_P, _P, _I, _IP]),
    "ttn_envs_create": (_I, [_P, _P, C.POINTER(_P)]),
    "ttn_envs_destroy": (None, [_P]),
    "ttn_env_update": (_I, [_P, _P, _P, _P, _I, _IP, _IP, _I, _P, _I]),
    "ttn_envs_get": (_I, [_P, _I, _I, _I, _DP, _LL]),
    "ttn_heff_apply": (_I, [_P, _P, _P, _I, _P, _P, _DP, _I]),
    "ttn_gram": (_I, [_P, _P, _P, _P, _DP, _DP, _I, _I, _I]),
    "ttn_apply_block": (_I, [_P, _P, _P, C.POINTER(_P), _I]),
    "ttn_recompress": (_I, [_P, _I, _DP, C.POINTER(_P), C.POINTER(_P), _IP, _P, _I, _I, _I]),
    "ttn_als_solve": (_I, [_P, _P, _DP, _P, _P, _I, _I, _D, _I]),
    "ttn_rayleigh_ritz": (_I, [_P, _I, _DP, _DP, _I, _D, _DP, _DP]),
    "ttn_lobpcg": (_I, [_P, _P, _P, _I, _D, _I, _I, _D, _I, _I, _DP]),
    "ttn_rayleigh_ritz_noalloc": (_I, [_P, _I, _P, _P, _I, _D, _P, _P]),
    "ttn_inverse_iteration": (_I, [_P, _P, _P, _I, _D, _I, _I, _D, _I, _I, _DP]),
    "ttn_src_apply": (_I, [_P, _P, _P, _I, _DP, C.POINTER(_P), _I]),
    "ttn_selftest_bounded_wait": (_I, [_P, _D]),
    "ttn_iteration_times": (_I, [_P, _DP, _I]),
    "ttn_ttno_rank_bounds": (_I, [_P, _IP]),
    "ttn_block_rayleigh_ritz": (_I, [_P, _P, _P, _D, _I, _I, _DP]),
    "ttn_fault_inject_alloc": (None, [_LL]),
}


class TTNError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def load():
    """Load libttn.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "paper_2512_15875_gb300.build.build()")
        lib = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


def exported_symbols():
    return list(_SIGS)


def _ip(a):
    return a.ctypes.data_as(_IP)


def _llp(a):
    return a.ctypes.data_as(_LLP)


def _dp(a):
    return None if a is None else a.ctypes.data_as(_DP)


def _prec(p):
    return PRECISION[p] if isinstance(p, str) else int(p)


# ----------------------------------------------------------------------------------------------
# handles
# ----------------------------------------------------------------------------------------------
_LIVE = weakref.WeakValueDictionary()   # live handles, for an ordered release at exit
_ORDER = {"ttn_envs_destroy": 0, "ttn_block_destroy": 1, "ttn_ttno_destroy": 2,
          "ttn_tree_destroy": 3, "ttn_destroy": 4}


def _release_all():
    """Destroy every live handle before the interpreter (and the CUDA runtime) shuts down:
    environments and blocks first, contexts last."""
    for h in sorted(list(_LIVE.values()), key=lambda h: _ORDER.get(h._destroy, 9)):
        try:
            h.close()
        except Exception:
            pass


atexit.register(_release_all)


class _Handle:
    _destroy = None

    def __init__(self, ptr, ctx=None):
        self.ptr = ptr
        self.ctx = ctx
        _LIVE[id(self)] = self

    def close(self):
        if self.ptr:
            getattr(load(), self._destroy)(self.ptr)
            self.ptr = None
        _LIVE.pop(id(self), None)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def _as_parameter_(self):
        return self.ptr


class Context(_Handle):
    _destroy = "ttn_destroy"

    def check(self, st):
        if st != 0:
            msg = load().ttn_last_error(self.ptr).decode()
            raise TTNError(st, msg)
        return st


class Tree(_Handle):
    _destroy = "ttn_tree_destroy"


class TTNO(_Handle):
    _destroy = "ttn_ttno_destroy"


class Block(_Handle):
    _destroy = "ttn_block_destroy"


class Envs(_Handle):
    _destroy = "ttn_envs_destroy"


# ----------------------------------------------------------------------------------------------
# entry points (same names as the C ABI)
# ----------------------------------------------------------------------------------------------
def ttn_create(device=0, stream=None) -> Context:
    lib = load()
    p = _P()
    st = lib.ttn_create(C.byref(p), int(device), stream)
    if st != 0:
        raise TTNError(st, "ttn_create failed")
    return Context(p.value)


def ttn_selftest_bounded_wait(ctx, budget_ms=1.0):
    """Returns the status of a barrier wait that is made to run out (TTN_ETIMEOUT = 6)."""
    return load().ttn_selftest_bounded_wait(ctx.ptr, float(budget_ms))


def ttn_iteration_times(ctx, max_n=100000):
    """ms from the start of the last ttn_lobpcg / ttn_inverse_iteration call to the end of each
    iteration (index 0: the initial Rayleigh quotients)."""
    out = np.zeros(max_n)
    n = load().ttn_iteration_times(ctx.ptr, _dp(out), int(max_n))
    if n < 0:
        raise TTNError(3, "ttn_iteration_times: CUDA error")
    return out[:min(n, max_n)]


def ttn_fault_inject_alloc(after):
    load().ttn_fault_inject_alloc(int(after))


def ttn_synchronize(ctx):
    ctx.check(load().ttn_synchronize(ctx.ptr))


def ttn_launch_count(ctx) -> int:
    return int(load().ttn_launch_count(ctx.ptr))


def ttn_flop_count(ctx) -> float:
    return float(load().ttn_flop_count(ctx.ptr))


def ttn_profile_enable(ctx, on=True):
    ctx.check(load().ttn_profile_enable(ctx.ptr, 1 if on else 0))


def ttn_profile_get(ctx, max_kernels=64):
    """{kernel name: dict(launches, ms, flops, bytes)} since the last ttn_profile_enable."""
    names = C.create_string_buffer(64 * max_kernels)
    launches = np.zeros(max_kernels, dtype=np.int64)
    ms, fl, by = np.zeros(max_kernels), np.zeros(max_kernels), np.zeros(max_kernels)
    nk = C.c_int()
    ctx.check(load().ttn_profile_get(ctx.ptr, max_kernels, names, _llp(launches), _dp(ms),
                                     _dp(fl), _dp(by), C.byref(nk)))
    out = {}
    for i in range(min(nk.value, max_kernels)):
        nm = names.raw[64 * i:64 * i + 64].split(b"\0")[0].decode()
        out[nm] = dict(launches=int(launches[i]), ms=float(ms[i]), flops=float(fl[i]),
                       bytes=float(by[i]))
    return out


def ttn_tree_create(ctx, tree) -> Tree:
    """``tree``: an object with ``parent`` and ``phys_dim`` arrays."""
    parent = np.ascontiguousarray(tree.parent, dtype=np.int32)
    phys = np.ascontiguousarray(tree.phys_dim, dtype=np.int32)
    p = _P()
    ctx.check(load().ttn_tree_create(ctx.ptr, len(parent), _ip(parent), _ip(phys), C.byref(p)))
    t = Tree(p.value, ctx)
    t.n_nodes = len(parent)
    return t


def ttn_build_ttno(ctx, tree_h, flat, tol=1e-12):
    """``flat``: the dict of ``inputs.Hamiltonian.flat(tree)``. Returns (TTNO, bond dims)."""
    lib = load()
    f = {k: np.ascontiguousarray(v) for k, v in flat.items()}
    bonds = np.zeros(tree_h.n_nodes, dtype=np.int32)
    p = _P()
    ctx.check(lib.ttn_build_ttno(
        ctx.ptr, tree_h.ptr, len(f["op_site"]), _ip(f["op_site"].astype(np.int32)),
        _llp(f["op_offset"].astype(np.int64)), _dp(f["op_data"].astype(np.float64)),
        len(f["coeff"]), _dp(f["coeff"].astype(np.float64)),
        _ip(f["term_offset"].astype(np.int32)), _ip(f["term_op_ids"].astype(np.int32)),
        float(tol), C.byref(p), _ip(bonds)))
    return TTNO(p.value, ctx), bonds


def ttn_ttno_rank_bounds(H, n_nodes):
    """Per edge: the smallest operator bond an exact TTNO can have (numerical rank of the
    coefficient matrix across the edge); -1 where unknown."""
    out = np.zeros(n_nodes, dtype=np.int32)
    H.ctx.check(load().ttn_ttno_rank_bounds(H.ptr, _ip(out)))
    return out


def ttn_ttno_create(ctx, tree_h, wbond, ops, entries):
    """ops: list of (node, d x d array); entries: list of (node, w tuple, op index, coef)."""
    wbond = np.ascontiguousarray(wbond, dtype=np.int32)
    op_site = np.array([n for n, _ in ops], dtype=np.int32)
    op_off = np.zeros(len(ops) + 1, dtype=np.int64)
    op_off[1:] = np.cumsum([np.asarray(m).size for _, m in ops])
    op_data = (np.concatenate([np.asarray(m, dtype=np.float64).ravel() for _, m in ops])
               if ops else np.zeros(1))
    ne = len(entries)
    en = np.array([e[0] for e in entries], dtype=np.int32)
    ew = np.zeros((max(ne, 1), TTN_MAX_LEGS), dtype=np.int32)
    for i, e in enumerate(entries):
        ew[i, :len(e[1])] = e[1]
    eo = np.array([e[2] for e in entries], dtype=np.int32)
    ec = np.array([e[3] for e in entries], dtype=np.float64)
    p = _P()
    ctx.check(load().ttn_ttno_create(ctx.ptr, tree_h.ptr, _ip(wbond), len(ops), _ip(op_site),
                                     _llp(op_off), _dp(op_data), ne, _ip(en), _ip(ew), _ip(eo),
                                     _dp(ec), C.byref(p)))
    return TTNO(p.value, ctx)


def ttn_ttno_info(H, n_nodes):
    wb = np.zeros(n_nodes, dtype=np.int32)
    ne = C.c_int()
    nd = C.c_longlong()
    H.ctx.check(load().ttn_ttno_info(H.ptr, _ip(wb), C.byref(ne), C.byref(nd)))
    return wb, ne.value, nd.value


def ttn_ttno_get_entries(H, n_nodes):
    """Returns (wbond, list of (node, w tuple (TTN_MAX_LEGS), coef, d x d op))."""
    wb, ne, nd = ttn_ttno_info(H, n_nodes)
    node = np.zeros(max(ne, 1), dtype=np.int32)
    w = np.zeros((max(ne, 1), TTN_MAX_LEGS), dtype=np.int32)
    coef = np.zeros(max(ne, 1))
    off = np.zeros(ne + 1, dtype=np.int64)
    data = np.zeros(max(nd, 1))
    H.ctx.check(load().ttn_ttno_get_entries(H.ptr, _ip(node), _ip(w), _dp(coef), _llp(off),
                                            _dp(data)))
    out = []
    for e in range(ne):
        blk = data[off[e]:off[e + 1]]
        d = int(round(np.sqrt(blk.size)))
        out.append((int(node[e]), tuple(w[e]), float(coef[e]), blk.reshape(d, d)))
    return wb, out


def ttn_block_create(ctx, tree_h, n_states, bonds) -> Block:
    bonds = np.ascontiguousarray(bonds, dtype=np.int32)
    p = _P()
    ctx.check(load().ttn_block_create(ctx.ptr, tree_h.ptr, int(n_states), _ip(bonds),
                                      C.byref(p)))
    b = Block(p.value, ctx)
    b.n_states = int(n_states)
    b.n_nodes = tree_h.n_nodes
    return b


def ttn_block_set(b, state, node, arr):
    a = np.ascontiguousarray(arr, dtype=np.float64)
    b.ctx.check(load().ttn_block_set(b.ptr, int(state), int(node), _dp(a), a.size))


def ttn_block_node_info(b, node):
    sz = C.c_longlong()
    dp = _DP()
    b.ctx.check(load().ttn_block_node_info(b.ptr, int(node), C.byref(sz), C.byref(dp)))
    return sz.value, C.cast(dp, C.c_void_p).value


def ttn_block_get(b, state, node, shape=None):
    sz, _ = ttn_block_node_info(b, node)
    n = sz * (b.n_states if state < 0 else 1)
    out = np.zeros(n)
    b.ctx.check(load().ttn_block_get(b.ptr, int(state), int(node), _dp(out), n))
    return out if shape is None else out.reshape(shape)


def ttn_block_copy_states(dst, src, src_states):
    s = np.ascontiguousarray(src_states, dtype=np.int32)
    dst.ctx.check(load().ttn_block_copy_states(dst.ptr, src.ptr, len(s), _ip(s)))


def ttn_envs_create(ctx, tree_h) -> Envs:
    p = _P()
    ctx.check(load().ttn_envs_create(ctx.ptr, tree_h.ptr, C.byref(p)))
    return Envs(p.value, ctx)


def ttn_env_update(ctx, H, bra, ket, pair_bra, pair_ket, direction, envs, prec="fp64"):
    pb = np.ascontiguousarray(pair_bra, dtype=np.int32)
    pk = np.ascontiguousarray(pair_ket, dtype=np.int32)
    ctx.check(load().ttn_env_update(ctx.ptr, H.ptr if H is not None else None, bra.ptr, ket.ptr,
                                    len(pb), _ip(pb), _ip(pk), int(direction), envs.ptr,
                                    _prec(prec)))


def ttn_envs_get(envs, node, direction, pair, shape):
    out = np.zeros(int(np.prod(shape)))
    envs.ctx.check(load().ttn_envs_get(envs.ptr, int(node), int(direction), int(pair), _dp(out),
                                       out.size))
    return out.reshape(shape)


def ttn_heff_apply(ctx, H, envs, node, x, y, shift=None, prec="fp64"):
    s = None if shift is None else np.ascontiguousarray(shift, dtype=np.float64)
    ctx.check(load().ttn_heff_apply(ctx.ptr, H.ptr, envs.ptr, int(node), x.ptr, y.ptr, _dp(s),
                                    _prec(prec)))


def ttn_gram(ctx, H, bra, ket, want_s=True, want_h=True, prec="fp64"):
    """Returns (S, Hm) host matrices (None where not requested)."""
    nb, nk = bra.n_states, ket.n_states
    S = np.zeros((nb, nk)) if want_s else None
    Hm = np.zeros((nb, nk)) if want_h else None
    ctx.check(load().ttn_gram(ctx.ptr, H.ptr if H is not None else None, bra.ptr, ket.ptr,
                              _dp(S), _dp(Hm), nk, 0, _prec(prec)))
    return S, Hm


def ttn_gram_device(ctx, H, bra, ket, S_ptr, H_ptr, ld, prec="fp64"):
    """Device-output variant: S_ptr/H_ptr are device addresses (ints) or None."""
    ctx.check(load().ttn_gram(ctx.ptr, H.ptr if H is not None else None, bra.ptr, ket.ptr,
                              C.cast(S_ptr, _DP) if S_ptr else None,
                              C.cast(H_ptr, _DP) if H_ptr else None, int(ld), 1, _prec(prec)))


def ttn_apply_block(ctx, H, block, prec="fp64") -> Block:
    p = _P()
    ctx.check(load().ttn_apply_block(ctx.ptr, H.ptr, block.ptr, C.byref(p), _prec(prec)))
    b = Block(p.value, ctx)
    b.n_states = block.n_states
    b.n_nodes = block.n_nodes
    return b


def ttn_src_apply(ctx, H, x, chi, omega, prec="fp64") -> Block:
    """omega: per-node d_i x chi matrices (None for auxiliary nodes), as inputs.src_sketch
    draws them. Returns the new block (bonds min(chi, d_i * prod of children's bonds))."""
    flat = np.ascontiguousarray(np.concatenate(
        [np.asarray(o, dtype=np.float64).ravel() for o in omega if o is not None]))
    p = _P()
    ctx.check(load().ttn_src_apply(ctx.ptr, H.ptr, x.ptr, int(chi), _dp(flat), C.byref(p),
                                   _prec(prec)))
    b = Block(p.value, ctx)
    b.n_states = x.n_states
    b.n_nodes = x.n_nodes
    return b


def ttn_recompress(ctx, coeff, ops, blocks, in_state, out, n_sweeps=2, prec="fp64"):
    """coeff: (n_in, n_out) array; ops/blocks: per-input TTNO (or None) and Block."""
    coeff = np.ascontiguousarray(coeff, dtype=np.float64)
    n_in, n_out = coeff.shape
    op_arr = (C.c_void_p * n_in)(*[o.ptr if o is not None else None for o in ops])
    bl_arr = (C.c_void_p * n_in)(*[b.ptr for b in blocks])
    st = np.ascontiguousarray(in_state, dtype=np.int32)
    ctx.check(load().ttn_recompress(ctx.ptr, n_in, _dp(coeff), op_arr, bl_arr, _ip(st), out.ptr,
                                    n_out, int(n_sweeps), _prec(prec)))


def ttn_als_solve(ctx, H, shift, rhs, y, n_sweeps=2, minres_max=10, minres_tol=1e-5,
                  prec="fp64"):
    s = np.ascontiguousarray(shift, dtype=np.float64)
    st = load().ttn_als_solve(ctx.ptr, H.ptr, _dp(s), rhs.ptr, y.ptr, int(n_sweeps),
                              int(minres_max), float(minres_tol), _prec(prec))
    if st not in (0, 5):
        ctx.check(st)
    return st


def ttn_rayleigh_ritz(ctx, Ht, Mt, n, eps=1e-12):
    Ht = np.ascontiguousarray(Ht, dtype=np.float64)
    Mt = np.ascontiguousarray(Mt, dtype=np.float64)
    m = Ht.shape[0]
    theta = np.zeros(n)
    V = np.zeros((m, n))
    ctx.check(load().ttn_rayleigh_ritz(ctx.ptr, m, _dp(Ht), _dp(Mt), int(n), float(eps),
                                       _dp(theta), _dp(V)))
    return theta, V


def ttn_rayleigh_ritz_noalloc(ctx, m, Ht_ptr, Mt_ptr, n, eps, theta_ptr, V_ptr):
    """Device-pointer variant that allocates no device memory (see include/ttn.h). All four
    pointers are device addresses (ints) owned by the caller. Returns the status: 0, or 5
    (TTN_ENOTCONV, results written) when an eigensolve stopped short of convergence."""
    st = load().ttn_rayleigh_ritz_noalloc(ctx.ptr, int(m), Ht_ptr, Mt_ptr, int(n), float(eps),
                                          theta_ptr, V_ptr)
    if st not in (0, 5):
        ctx.check(st)
    return st


def ttn_block_rayleigh_ritz(ctx, H, x, eps=1e-12, fit_sweeps=2, prec="fp64"):
    """Hc = ESc over all states of x (x is replaced by the fitted Ritz vectors); returns the
    Ritz values."""
    theta = np.zeros(x.n_states)
    ctx.check(load().ttn_block_rayleigh_ritz(ctx.ptr, H.ptr, x.ptr, float(eps), int(fit_sweeps),
                                             _prec(prec), _dp(theta)))
    return theta


def ttn_lobpcg(ctx, H, x, n_iter, shift_offset, als_sweeps=2, minres_max=10, minres_tol=1e-5,
               fit_sweeps=2, prec="fp64"):
    hist = np.zeros((n_iter + 1, x.n_states))
    st = load().ttn_lobpcg(ctx.ptr, H.ptr, x.ptr, int(n_iter), float(shift_offset),
                           int(als_sweeps), int(minres_max), float(minres_tol), int(fit_sweeps),
                           _prec(prec), _dp(hist))
    if st not in (0, 5):
        ctx.check(st)
    return hist


def ttn_inverse_iteration(ctx, H, x, n_iter, cluster_gap=0.0, als_sweeps=1, minres_max=10000,
                          minres_tol=1e-5, fit_sweeps=2, prec="fp64"):
    hist = np.zeros((n_iter + 1, x.n_states))
    st = load().ttn_inverse_iteration(ctx.ptr, H.ptr, x.ptr, int(n_iter), float(cluster_gap),
                                      int(als_sweeps), int(minres_max), float(minres_tol),
                                      int(fit_sweeps), _prec(prec), _dp(hist))
    if st not in (0, 5):
        ctx.check(st)
    return hist


# ----------------------------------------------------------------------------------------------
# conveniences (marshalling only)
# ----------------------------------------------------------------------------------------------
def block_from_arrays(ctx, tree_h, bonds, arrays) -> Block:
    """arrays[node] of shape (n_states, *node_shape) -> device block."""
    n = arrays[0].shape[0]
    b = ttn_block_create(ctx, tree_h, n, bonds)
    for t, a in enumerate(arrays):
        ttn_block_set(b, -1, t, a)
    return b


def block_to_arrays(b, shapes):
    return [ttn_block_get(b, -1, t).reshape((b.n_states,) + tuple(shapes[t]))
            for t in range(b.n_nodes)]
