"""ctypes binding of libsph.so (include/sph.h): argument marshalling only.

Every function has the C name and raises :class:`SphError` with the library's
message when the status is not SPH_OK.  Device pointers are plain integers
(e.g. ``tensor.data_ptr()``); streams are ``torch.cuda.Stream.cuda_stream``
integers or 0.  There is no fallback: if the library is missing, importing
fails loudly.
"""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
# SPH_CHECKED_BUILD=1 selects the index-checked build (python -m
# paper_2606_23891_b300.build --check), for tests of the kernels' bounds.
LIB_PATH = os.path.join(_HERE, "libsph_check.so" if os.environ.get("SPH_CHECKED_BUILD") == "1"
                        else "libsph.so")

SPH_AOS, SPH_AOS_RANDOM, SPH_SAOS_PACK_GRAD, SPH_SAOS_PACK_FORCE, \
    SPH_SAOS_PACK_SHARED, SPH_SAOS_PACK_GRAD_TYPE, SPH_SAOS_PACK_FORCE_TYPE, \
    SPH_SAOS_PACK_SHARED_TYPE, SPH_SOA, SPH_SAOS_PACK_FORCE_REPL, SPH_SAOS_FUSED = range(11)
LAYOUTS = {"aos": 0, "aos_random": 1, "pack_grad": 2, "pack_force": 3,
           "pack_shared": 4, "pack_grad_type": 5, "pack_force_type": 6,
           "pack_shared_type": 7, "soa": 8, "pack_force_repl": 9, "fused": 10}
SPH_DENSITY, SPH_GRADIENT, SPH_FORCE = 0, 1, 2
LOOPS = {"density": 0, "gradient": 1, "force": 2}
STATUS = {0: "SPH_OK", 1: "SPH_EINVAL", 2: "SPH_ENOMEM", 3: "SPH_ECUDA",
          4: "SPH_EBOUNDS", 5: "SPH_ETIMEOUT", 6: "SPH_EUNSUPPORTED"}

FIELD_NAMES = ("x", "v", "a", "mass", "h", "u", "u_dt", "rho", "time_bin",
               "alpha_visc", "alpha_diff", "rho_dh", "wcount", "wcount_dh",
               "div_v", "rot_v", "f_gradh", "pressure", "soundspeed", "balsara",
               "v_sig_grad", "laplace_u", "h_dt", "v_sig", "id")


class SphError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s: %s" % (STATUS.get(status, status), msg))
        self.status = status


class Fields(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in FIELD_NAMES]


class Params(C.Structure):
    _fields_ = [("gamma", C.c_double), ("kernel_gamma", C.c_double),
                ("beta_visc", C.c_double), ("balsara_eps", C.c_double),
                ("active_bin", C.c_int32), ("reserved", C.c_int32)]


class GridParams(C.Structure):
    _fields_ = [("box", C.c_double * 3), ("kernel_gamma", C.c_double),
                ("ncell", C.c_int32 * 3), ("reserved", C.c_int32),
                ("bundle_max_slots", C.c_int64)]


class BatchParams(C.Structure):
    _fields_ = [("max_target_cells", C.c_int64), ("threads", C.c_int32),
                ("reserved", C.c_int32)]


class TreeParams(C.Structure):
    _fields_ = [("box", C.c_double * 3), ("kernel_gamma", C.c_double),
                ("leaf_max", C.c_int32), ("rule", C.c_int32)]


def params(gamma=5.0 / 3.0, kernel_gamma=1.825742, beta_visc=3.0,
           balsara_eps=1e-4, active_bin=0) -> Params:
    return Params(gamma, kernel_gamma, beta_visc, balsara_eps, active_bin, 0)


def grid_params(box=(1.0, 1.0, 1.0), kernel_gamma=1.825742, ncell=(0, 0, 0),
                bundle_max_slots=0) -> GridParams:
    g = GridParams()
    g.box[:] = list(box)
    g.kernel_gamma = kernel_gamma
    g.ncell[:] = list(ncell)
    g.reserved = 0
    g.bundle_max_slots = bundle_max_slots
    return g


_lib = None


def lib() -> C.CDLL:
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError("%s is not built; run `python -m paper_2606_23891_b300.build%s`"
                          % (os.path.basename(LIB_PATH),
                             " --check" if LIB_PATH.endswith("_check.so") else ""))
    L = C.CDLL(LIB_PATH)
    p, i, i64, u64, sz = C.c_void_p, C.c_int, C.c_int64, C.c_uint64, C.c_size_t
    sig = {
        "sph_version": (C.c_char_p, []),
        "sph_last_error": (C.c_char_p, []),
        "sph_store_bytes": (sz, [i64, i, u64]),
        "sph_layout_group_count": (i, [i, u64]),
        "sph_layout_describe": (i, [i, u64, i, p, p, p, p, p]),
        "sph_store_create": (i, [i64, i, u64, p, sz, p]),
        "sph_store_destroy": (i, [p]),
        "sph_store_import": (i, [p, p, p, p]),
        "sph_store_export": (i, [p, p, p, p]),
        "sph_store_convert": (i, [p, p, p]),
        "sph_fault_inject": (i, [i, i]),
        "sph_pack_host_fission": (i, [p, p, i, i, p, i, i]),
        "sph_unpack_host_fission": (i, [p, p, i, i, p, i, i]),
        "sph_tasks_build": (i, [i64, p, p, p, p, p]),
        "sph_tasks_upload": (i, [p]),
        "sph_tasks_info": (i, [p, p]),
        "sph_tasks_get": (i, [p, p, p, p, p, p]),
        "sph_buffer_bytes": (sz, [p, i, i]),
        "sph_init": (i, [p, i, p, p]),
        "sph_pack": (i, [p, p, i, i, p, p]),
        "sph_density": (i, [p, i, p, p, p, p]),
        "sph_gradient": (i, [p, i, p, p, p, p]),
        "sph_force": (i, [p, i, p, p, p, p]),
        "sph_unpack": (i, [p, p, i, i, p, p]),
        "sph_ghost": (i, [p, i, p, p]),
        "sph_offload_loop": (i, [p, p, i, p, p, p, p]),
        "sph_count_pairs": (i, [p, i, i, p, p, p, p]),
        "sph_sync": (i, [p]),
        "sph_offload_loop_noalloc": (i, [p, p, i, p, p]),
        "sph_batch_build": (i, [p, p, p]),
        "sph_batch_info": (i, [p, p]),
        "sph_batch_buffer_bytes": (sz, [p, i, i]),
        "sph_batch_pack": (i, [p, p, i, i, p, p, p]),
        "sph_batch_pack_list": (i, [p, p, i, i, p, p, p]),
        "sph_batch_interact": (i, [p, i, i, p, p, p, p]),
        "sph_batch_unpack": (i, [p, p, i, i, p, p, p]),
        "sph_batch_unpack_write": (i, [p, p, i, i, p, p, p, i, p]),
        "sph_batch_offload_loop": (i, [p, p, i, p, p, p, p]),
        "sph_batch_destroy": (i, [p]),
        "sph_batch_buffer_bytes_fp64": (sz, [p, i]),
        "sph_batch_build_tree": (i, [i64, p, p, p, p, p, p]),
        "sph_batch_plan_info": (i, [p, p]),
        "sph_batch_cells": (i, [p, i, p, p]),
        "sph_batch_list_bytes": (sz, [p, i64]),
        "sph_batch_list_build": (i, [p, p, p, p, sz, p, p]),
        "sph_batch_list_build_bundle": (i, [p, p, i, p, p, sz, p, p]),
        "sph_batch_list_fixed": (i, [p]),
        "sph_batch_list_status": (i, [p, p, p]),
        "sph_batch_list_count": (i, [p, p, i, p, p, sz, p, p, p]),
        "sph_batch_list_symmetric": (i, [p, i]),
        "sph_batch_offload_loop_list": (i, [p, p, i, p, p, p, sz, p, p]),
        "sph_batch_offload_step_list": (i, [p, p, p, p, p, sz, p, p]),
        "sph_batch_list_interact": (i, [p, i, i, p, p, p, sz, p, p]),
        "sph_batch_adjoint_bytes": (sz, [p]),
        "sph_batch_x64_bytes": (sz, [p]),
        "sph_batch_offload_step_list_x64": (i, [p, p, p, p, p, sz, p, sz, p, p]),
        "sph_batch_offload_loop_host": (i, [p, p, i, p, p, p, p, p, p, i]),
        "sph_batch_adjoint": (i, [p, p, p, p, sz, p, sz, p, p, p, p, p, p, p, p]),
        "sph_tree_plan": (i, [i64, p, p, p, p, p, p, p, p, i64, p]),
        "sph_batch_count_pairs": (i, [p, p, i, p, p, p, p]),
        "sph_batch_offload_loop_fp64": (i, [p, p, i, p, p, p, p]),
        "sph_store_create_host": (i, [i64, i, u64, p, sz, p]),
        "sph_store_import_host": (i, [p, p, p, i]),
        "sph_store_export_host": (i, [p, p, p, i]),
        "sph_pack_host": (i, [p, p, i, i, p, i]),
        "sph_unpack_host": (i, [p, p, i, i, p, i]),
        "sph_init_host": (i, [p, i, p, i]),
        "sph_ghost_host": (i, [p, i, p, i]),
        "sph_offload_loop_host": (i, [p, p, i, p, p, p, p, p, p, i]),
        "sph_offload_loop_host_stats": (i, [p, p, i, p, p, p, p, p, p, i, p]),
        "sph_hostio_bytes": (sz, [i64, p, p]),
        "sph_hostio_create": (i, [p, p, p, p, p, sz, p, p, p]),
        "sph_hostio_begin": (i, [p, p, p]),
        "sph_hostio_end": (i, [p, p, p]),
        "sph_hostio_drain": (i, [p, p]),
        "sph_hostio_info": (i, [p, p]),
        "sph_hostio_destroy": (i, [p]),
        "sph_peak_run": (i, [i, i64, p, p, p]),
        "sph_tasks_destroy": (i, [p]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def _ok(rc: int) -> None:
    if rc != 0:
        raise SphError(rc, lib().sph_last_error().decode())


def sph_version() -> str:
    return lib().sph_version().decode()


def sph_last_error() -> str:
    return lib().sph_last_error().decode()


def sph_store_bytes(n: int, layout: int, seed: int = 0) -> int:
    return lib().sph_store_bytes(n, layout, seed)


def sph_layout_group_count(layout: int, seed: int = 0) -> int:
    return lib().sph_layout_group_count(layout, seed)


def sph_layout_describe(layout: int, seed: int, group: int):
    """(record_bytes, [(field_id, comp, offset), ...])"""
    nm = C.c_int32()
    fl, co, of = (C.c_int32 * 32)(), (C.c_int32 * 32)(), (C.c_int32 * 32)()
    rec = C.c_int32()
    _ok(lib().sph_layout_describe(layout, seed, group, C.byref(nm), fl, co, of,
                                  C.byref(rec)))
    return rec.value, [(fl[k], co[k], of[k]) for k in range(nm.value)]


def sph_store_create(n: int, layout: int, seed: int, dev_mem: int, nbytes: int):
    h = C.c_void_p()
    _ok(lib().sph_store_create(n, layout, seed, dev_mem, nbytes, C.byref(h)))
    return h


def sph_store_destroy(s) -> None:
    _ok(lib().sph_store_destroy(s))


def sph_store_import(s, fields: Fields, dev_perm: int, stream: int = 0) -> None:
    _ok(lib().sph_store_import(s, C.byref(fields), dev_perm, stream))


def sph_store_export(s, fields: Fields, dev_perm: int, stream: int = 0) -> None:
    _ok(lib().sph_store_export(s, C.byref(fields), dev_perm, stream))


FISSION = {"none": 0, "by_struct": 1, "by_element": 2, "by_type": 3, "by_struct_and_type": 4}


def sph_pack_host_fission(s, t, loop: int, bundle: int, host_buf: int, fission: int,
                          nthreads: int = 0) -> None:
    _ok(lib().sph_pack_host_fission(s, t, loop, bundle, host_buf, fission, nthreads))


def sph_unpack_host_fission(s, t, loop: int, bundle: int, host_buf: int, fission: int,
                            nthreads: int = 0) -> None:
    _ok(lib().sph_unpack_host_fission(s, t, loop, bundle, host_buf, fission, nthreads))


SPH_FAULT_NONE, SPH_FAULT_DEVICE_ALLOC, SPH_FAULT_COPY = 0, 1, 2


def sph_fault_inject(site: int, countdown: int) -> None:
    _ok(lib().sph_fault_inject(site, countdown))


def sph_store_convert(dst, src, stream: int = 0) -> None:
    _ok(lib().sph_store_convert(dst, src, stream))


def sph_tasks_build(n: int, host_x: int, host_h: int, gp: GridParams,
                    host_perm_out: int):
    h = C.c_void_p()
    _ok(lib().sph_tasks_build(n, host_x, host_h, C.byref(gp), host_perm_out,
                              C.byref(h)))
    return h


def sph_tasks_upload(t) -> None:
    _ok(lib().sph_tasks_upload(t))


def sph_tasks_info(t) -> dict:
    info = (C.c_int64 * 10)()
    _ok(lib().sph_tasks_info(t, info))
    keys = ("ncell_x", "ncell_y", "ncell_z", "ntasks", "nbundles", "slots",
            "max_bundle_slots", "nonempty_cells", "n", "max_cell")
    return dict(zip(keys, list(info)))


def sph_tasks_get(t, ci=0, cj=0, shift=0, cell_start=0, bundle_start=0) -> None:
    _ok(lib().sph_tasks_get(t, ci or None, cj or None, shift or None,
                            cell_start or None, bundle_start or None))


def sph_buffer_bytes(t, loop: int, in_or_out: int) -> int:
    return lib().sph_buffer_bytes(t, loop, in_or_out)


def sph_init(s, loop: int, p: Params, stream: int = 0) -> None:
    _ok(lib().sph_init(s, loop, C.byref(p), stream))


def sph_pack(s, t, loop: int, bundle: int, dev_buf_in: int, stream: int = 0) -> None:
    _ok(lib().sph_pack(s, t, loop, bundle, dev_buf_in, stream))


def sph_density(t, bundle: int, dev_in: int, dev_out: int, p: Params, stream: int = 0):
    _ok(lib().sph_density(t, bundle, dev_in, dev_out, C.byref(p), stream))


def sph_gradient(t, bundle: int, dev_in: int, dev_out: int, p: Params, stream: int = 0):
    _ok(lib().sph_gradient(t, bundle, dev_in, dev_out, C.byref(p), stream))


def sph_force(t, bundle: int, dev_in: int, dev_out: int, p: Params, stream: int = 0):
    _ok(lib().sph_force(t, bundle, dev_in, dev_out, C.byref(p), stream))


def sph_unpack(s, t, loop: int, bundle: int, dev_buf_out: int, stream: int = 0) -> None:
    _ok(lib().sph_unpack(s, t, loop, bundle, dev_buf_out, stream))


def sph_ghost(s, after_loop: int, p: Params, stream: int = 0) -> None:
    _ok(lib().sph_ghost(s, after_loop, C.byref(p), stream))


def sph_offload_loop(s, t, loop: int, dev_in: int, dev_out: int, p: Params,
                     stream: int = 0) -> None:
    _ok(lib().sph_offload_loop(s, t, loop, dev_in, dev_out, C.byref(p), stream))


def sph_count_pairs(t, loop: int, bundle: int, dev_in: int, p: Params,
                    dev_count: int, stream: int = 0) -> None:
    _ok(lib().sph_count_pairs(t, loop, bundle, dev_in, C.byref(p), dev_count, stream))


SPH_NOALLOC_SCRATCH_BYTES = 32 << 20


def sph_offload_loop_noalloc(s, t, loop: int, p: Params, stream: int = 0) -> None:
    """sph_offload_loop with the library's own fixed scratch array instead of
    caller buffers; allocates nothing (see include/sph.h for the limits)."""
    _ok(lib().sph_offload_loop_noalloc(s, t, loop, C.byref(p), stream))


def sph_store_create_host(n: int, layout: int, seed: int, host_mem: int, nbytes: int):
    h = C.c_void_p()
    _ok(lib().sph_store_create_host(n, layout, seed, host_mem, nbytes, C.byref(h)))
    return h


def sph_store_import_host(s, fields: Fields, host_perm: int, nthreads: int = 0) -> None:
    _ok(lib().sph_store_import_host(s, C.byref(fields), host_perm, nthreads))


def sph_store_export_host(s, fields: Fields, host_perm: int, nthreads: int = 0) -> None:
    _ok(lib().sph_store_export_host(s, C.byref(fields), host_perm, nthreads))


def sph_pack_host(s, t, loop: int, bundle: int, host_buf_in: int, nthreads: int = 0) -> None:
    _ok(lib().sph_pack_host(s, t, loop, bundle, host_buf_in, nthreads))


def sph_unpack_host(s, t, loop: int, bundle: int, host_buf_out: int, nthreads: int = 0) -> None:
    _ok(lib().sph_unpack_host(s, t, loop, bundle, host_buf_out, nthreads))


def sph_init_host(s, loop: int, p: Params, nthreads: int = 0) -> None:
    _ok(lib().sph_init_host(s, loop, C.byref(p), nthreads))


def sph_ghost_host(s, after_loop: int, p: Params, nthreads: int = 0) -> None:
    _ok(lib().sph_ghost_host(s, after_loop, C.byref(p), nthreads))


def sph_offload_loop_host(s, t, loop: int, host_in, host_out, dev_in, dev_out, p: Params,
                          streams, nthreads: int = 0) -> None:
    """host_in, host_out, dev_in, dev_out, streams: pairs of pointers."""
    arr = lambda v: (C.c_void_p * 2)(*[int(x) for x in v])
    _ok(lib().sph_offload_loop_host(s, t, loop, arr(host_in), arr(host_out), arr(dev_in),
                                    arr(dev_out), C.byref(p), arr(streams), nthreads))


class StagedStats(C.Structure):
    _fields_ = [("wall_s", C.c_double), ("host_pack_s", C.c_double),
                ("host_unpack_s", C.c_double), ("host_wait_s", C.c_double),
                ("h2d_ms", C.c_double), ("kernel_ms", C.c_double), ("d2h_ms", C.c_double),
                ("h2d_bytes", C.c_int64), ("d2h_bytes", C.c_int64), ("bundles", C.c_int64)]


def sph_offload_loop_host_stats(s, t, loop: int, host_in, host_out, dev_in, dev_out,
                                p: Params, streams, nthreads: int = 0) -> dict:
    """sph_offload_loop_host with every stage timed; returns the stats."""
    arr = lambda v: (C.c_void_p * 2)(*[int(x) for x in v])
    st = StagedStats()
    _ok(lib().sph_offload_loop_host_stats(s, t, loop, arr(host_in), arr(host_out), arr(dev_in),
                                          arr(dev_out), C.byref(p), arr(streams), nthreads,
                                          C.byref(st)))
    return {name: getattr(st, name) for name, _ in StagedStats._fields_}


def sph_hostio_bytes(n: int, in_sel: Fields, out_sel: Fields) -> int:
    return lib().sph_hostio_bytes(n, C.byref(in_sel), C.byref(out_sel))


def sph_hostio_create(s, dev_perm: int, in_sel: Fields, out_sel: Fields, dev_staging: int,
                      nbytes: int, copy_in_stream: int, copy_out_stream: int):
    h = C.c_void_p()
    _ok(lib().sph_hostio_create(s, dev_perm, C.byref(in_sel), C.byref(out_sel), dev_staging,
                                nbytes, copy_in_stream, copy_out_stream, C.byref(h)))
    return h


def sph_hostio_begin(io, host_in: Fields, stream: int = 0) -> None:
    _ok(lib().sph_hostio_begin(io, C.byref(host_in), stream))


def sph_hostio_end(io, host_out: Fields, stream: int = 0) -> None:
    _ok(lib().sph_hostio_end(io, C.byref(host_out), stream))


def sph_hostio_drain(io, stream: int = 0) -> None:
    _ok(lib().sph_hostio_drain(io, stream))


def sph_hostio_info(io) -> dict:
    info = (C.c_int64 * 3)()
    _ok(lib().sph_hostio_info(io, info))
    return dict(zip(("h2d_bytes_per_step", "d2h_bytes_per_step", "steps"), list(info)))


def sph_hostio_destroy(io) -> None:
    _ok(lib().sph_hostio_destroy(io))


PEAK_FP32_FMA, PEAK_FP64_FMA, PEAK_FP64_ADD = 0, 1, 2


def sph_peak_run(kind: int, iters: int, dev_sink: int, stream: int = 0) -> float:
    """Launch one arithmetic-peak microbenchmark; returns its flop count."""
    fl = C.c_double()
    _ok(lib().sph_peak_run(kind, iters, dev_sink, stream, C.byref(fl)))
    return fl.value


def sph_batch_build(t, max_target_cells: int = 0, threads: int = 128):
    h = C.c_void_p()
    bp = BatchParams(max_target_cells, threads, 0)
    _ok(lib().sph_batch_build(t, C.byref(bp), C.byref(h)))
    return h


def sph_batch_build_tree(n: int, x_ptr: int, h_ptr: int, box=(1.0, 1.0, 1.0),
                         kernel_gamma=1.825742, leaf_max: int = 64,
                         max_target_cells: int = 0, threads: int = 128, perm_ptr: int = 0):
    h = C.c_void_p()
    tp = TreeParams()
    tp.box[:] = list(box)
    tp.kernel_gamma = kernel_gamma
    tp.leaf_max = leaf_max
    tp.rule = 0
    bp = BatchParams(max_target_cells, threads, 0)
    _ok(lib().sph_batch_build_tree(n, x_ptr, h_ptr, C.byref(tp), C.byref(bp), perm_ptr,
                                   C.byref(h)))
    return h


def sph_tree_plan(x, h, box=(1.0, 1.0, 1.0), kernel_gamma=1.825742, leaf_max: int = 64,
                  rule: int = 0):
    """Host-only tree plan: (perm, leaf_start, nb_start, nb) as numpy arrays."""
    import numpy as np
    x = np.ascontiguousarray(x, np.float64)
    h = np.ascontiguousarray(h, np.float32)
    n = x.shape[0]
    tp = TreeParams()
    tp.box[:] = list(box)
    tp.kernel_gamma = kernel_gamma
    tp.leaf_max = leaf_max
    tp.rule = rule
    perm = np.empty(n, np.int64)
    ls = np.empty(n + 1, np.int64)
    nbs = np.empty(n + 1, np.int64)
    nleaf, nnb = C.c_int64(), C.c_int64()
    args = (n, x.ctypes.data, h.ctypes.data, C.byref(tp), perm.ctypes.data, ls.ctypes.data,
            C.byref(nleaf), nbs.ctypes.data)
    rc = lib().sph_tree_plan(*args, None, 0, C.byref(nnb))
    if rc != 0 and nnb.value == 0:
        _ok(rc)
    nb = np.empty(max(nnb.value, 1), np.int32)
    _ok(lib().sph_tree_plan(*args, nb.ctypes.data, nb.size, C.byref(nnb)))
    L = nleaf.value
    return perm, ls[:L + 1].copy(), nbs[:L + 1].copy(), nb[:nnb.value].copy()


def sph_batch_plan_info(b) -> dict:
    info = (C.c_int64 * 4)()
    _ok(lib().sph_batch_plan_info(b, info))
    return dict(zip(("kind", "cells", "max_cell", "nbrs"), list(info)))


def sph_batch_cells(b, bundle: int):
    """(p0, n, slot) of every cell the bundle packs, an int32 array (ncells, 3)."""
    import numpy as np
    nc = C.c_int64()
    _ok(lib().sph_batch_cells(b, bundle, None, C.byref(nc)))
    out = np.empty((max(nc.value, 1), 3), np.int32)
    _ok(lib().sph_batch_cells(b, bundle, out.ctypes.data, C.byref(nc)))
    return out[:nc.value]


def sph_batch_count_pairs(s, b, loop: int, dev_in: int, p: Params, dev_count: int,
                          stream: int = 0):
    _ok(lib().sph_batch_count_pairs(s, b, loop, dev_in, C.byref(p), dev_count, stream))


def sph_batch_list_bytes(b, chunks: int) -> int:
    return lib().sph_batch_list_bytes(b, chunks)


def sph_batch_list_build(s, b, dev_in: int, dev_list: int, list_bytes: int, p: Params,
                         stream: int = 0):
    _ok(lib().sph_batch_list_build(s, b, dev_in, dev_list, list_bytes, C.byref(p), stream))


def sph_batch_list_build_bundle(s, b, bundle: int, dev_in: int, dev_list: int,
                                list_bytes: int, p: Params, stream: int = 0):
    _ok(lib().sph_batch_list_build_bundle(s, b, bundle, dev_in, dev_list, list_bytes,
                                          C.byref(p), stream))


def sph_batch_list_fixed(b) -> bool:
    r = lib().sph_batch_list_fixed(b)
    if r < 0:
        _ok(-r)
    return r == 1


def sph_batch_list_status(dev_list: int):
    need, ovf = C.c_int64(), C.c_int()
    _ok(lib().sph_batch_list_status(dev_list, C.byref(need), C.byref(ovf)))
    return need.value, ovf.value


def sph_batch_list_symmetric(b, enable: int = -1) -> bool:
    """Turn the symmetric list build on (1) / off (0) or ask (-1); returns
    whether later builds of the plan use it."""
    r = lib().sph_batch_list_symmetric(b, enable)
    if r < 0:
        _ok(-r)
    return r == 1


def sph_batch_list_count(s, b, bundle: int, dev_in: int, dev_list: int, list_bytes: int,
                         p: Params, dev_counts: int, stream: int = 0):
    _ok(lib().sph_batch_list_count(s, b, bundle, dev_in, dev_list, list_bytes, C.byref(p),
                                   dev_counts, stream))


def sph_batch_pack_list(s, b, loop: int, bundle: int, dev_in: int, p: Params, stream: int = 0):
    _ok(lib().sph_batch_pack_list(s, b, loop, bundle, dev_in, C.byref(p), stream))


def sph_batch_list_interact(b, loop: int, bundle: int, dev_in: int, dev_out: int, dev_list: int,
                            list_bytes: int, p: Params, stream: int = 0):
    _ok(lib().sph_batch_list_interact(b, loop, bundle, dev_in, dev_out, dev_list, list_bytes,
                                      C.byref(p), stream))


def sph_batch_offload_loop_host(s, b, loop: int, host_in, host_out, dev_in, dev_out,
                                p: Params, streams, nthreads: int = 0):
    arr = C.c_void_p * 2
    _ok(lib().sph_batch_offload_loop_host(s, b, loop, arr(*host_in), arr(*host_out),
                                          arr(*dev_in), arr(*dev_out), C.byref(p),
                                          arr(*streams), nthreads))


def sph_batch_x64_bytes(b) -> int:
    return lib().sph_batch_x64_bytes(b)


def sph_batch_offload_step_list_x64(s, b, dev_in: int, dev_out: int, dev_list: int,
                                    list_bytes: int, dev_x64: int, x64_bytes: int, p: Params,
                                    stream: int = 0):
    _ok(lib().sph_batch_offload_step_list_x64(s, b, dev_in, dev_out, dev_list, list_bytes,
                                              dev_x64, x64_bytes, C.byref(p), stream))


def sph_batch_adjoint_bytes(b) -> int:
    return lib().sph_batch_adjoint_bytes(b)


def sph_batch_adjoint(s, b, dev_in: int, dev_list: int, list_bytes: int, dev_scratch: int,
                      scratch_bytes: int, dev_store_perm: int, dev_abar: int, dev_ebar: int,
                      dev_gx: int, dev_gm: int, dev_gu: int, p: Params, stream: int = 0):
    _ok(lib().sph_batch_adjoint(s, b, dev_in, dev_list, list_bytes, dev_scratch, scratch_bytes,
                                dev_store_perm or None, dev_abar, dev_ebar, dev_gx, dev_gm,
                                dev_gu, C.byref(p), stream))


def sph_batch_offload_loop_list(s, b, loop: int, dev_in: int, dev_out: int, dev_list: int,
                                list_bytes: int, p: Params, stream: int = 0):
    _ok(lib().sph_batch_offload_loop_list(s, b, loop, dev_in, dev_out, dev_list, list_bytes,
                                          C.byref(p), stream))


def sph_batch_offload_step_list(s, b, dev_in: int, dev_out: int, dev_list: int,
                                list_bytes: int, p: Params, stream: int = 0):
    _ok(lib().sph_batch_offload_step_list(s, b, dev_in, dev_out, dev_list, list_bytes,
                                          C.byref(p), stream))


def sph_batch_info(b) -> dict:
    info = (C.c_int64 * 6)()
    _ok(lib().sph_batch_info(b, info))
    return dict(zip(("nbundles", "max_slots", "items", "threads", "max_targets", "cells"),
                    list(info)))


def sph_batch_buffer_bytes(b, loop: int, in_or_out: int) -> int:
    return lib().sph_batch_buffer_bytes(b, loop, in_or_out)


def sph_batch_pack(s, b, loop: int, bundle: int, dev_in: int, p: Params, stream: int = 0):
    _ok(lib().sph_batch_pack(s, b, loop, bundle, dev_in, C.byref(p), stream))


def sph_batch_interact(b, loop: int, bundle: int, dev_in: int, dev_out: int, p: Params,
                       stream: int = 0):
    _ok(lib().sph_batch_interact(b, loop, bundle, dev_in, dev_out, C.byref(p), stream))


def sph_batch_unpack(s, b, loop: int, bundle: int, dev_out: int, dev_in: int, stream: int = 0):
    _ok(lib().sph_batch_unpack(s, b, loop, bundle, dev_out, dev_in, stream))


def sph_batch_unpack_write(s, b, loop: int, bundle: int, dev_out: int, dev_in: int, p: Params,
                           with_ghost: int = 0, stream: int = 0):
    _ok(lib().sph_batch_unpack_write(s, b, loop, bundle, dev_out, dev_in, C.byref(p),
                                     with_ghost, stream))


def sph_batch_offload_loop(s, b, loop: int, dev_in: int, dev_out: int, p: Params,
                           stream: int = 0):
    _ok(lib().sph_batch_offload_loop(s, b, loop, dev_in, dev_out, C.byref(p), stream))


def sph_batch_buffer_bytes_fp64(b, in_or_out: int) -> int:
    return lib().sph_batch_buffer_bytes_fp64(b, in_or_out)


def sph_batch_offload_loop_fp64(s, b, loop: int, dev_in: int, dev_out: int, p: Params,
                                stream: int = 0):
    _ok(lib().sph_batch_offload_loop_fp64(s, b, loop, dev_in, dev_out, C.byref(p), stream))


def sph_batch_destroy(b) -> None:
    _ok(lib().sph_batch_destroy(b))


def sph_sync(stream: int = 0) -> None:
    _ok(lib().sph_sync(stream))


def sph_tasks_destroy(t) -> None:
    _ok(lib().sph_tasks_destroy(t))
