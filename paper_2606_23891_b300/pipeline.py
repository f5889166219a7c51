"""Drive the offload cycle of libsph over PyTorch-owned device memory.

PyTorch only provides device memory, pinned host memory and streams; every
step of the path (import into the store layout, pack, interaction kernels,
unpack, ghost, export) is a libsph call.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import sph

_TORCH_DT = {np.dtype(np.float64): torch.float64, np.dtype(np.float32): torch.float32,
             np.dtype(np.int8): torch.int8, np.dtype(np.int64): torch.int64}
_FIELD_DT = {"x": (np.float64, 3), "v": (np.float32, 3), "a": (np.float32, 3),
             "rot_v": (np.float32, 3), "time_bin": (np.int8, 1), "id": (np.int64, 1)}
INPUTS = ("x", "v", "mass", "h", "u", "alpha_visc", "alpha_diff", "time_bin", "id")
# the fields a step reads, and the results an integrator takes from it (the
# other outputs are intermediates that later loops of the same step consume)
STEP_INPUTS = ("x", "v", "mass", "h", "u", "alpha_visc", "alpha_diff", "time_bin")
STEP_RESULTS = ("rho", "a", "u_dt", "h_dt", "v_sig")
OUTPUTS = ("rho", "rho_dh", "wcount", "wcount_dh", "div_v", "rot_v", "f_gradh",
           "pressure", "soundspeed", "balsara", "v_sig_grad", "laplace_u", "a",
           "u_dt", "h_dt", "v_sig")


def field_spec(name: str):
    dt, k = _FIELD_DT.get(name, (np.float32, 1))
    return np.dtype(dt), k


def fields_struct(tensors: dict) -> sph.Fields:
    F = sph.Fields()
    for name, t in tensors.items():
        if t is None:
            continue
        if not t.is_contiguous():
            raise ValueError("field %s must be contiguous" % name)
        setattr(F, name, t.data_ptr())
    return F


class Offload:
    """One particle set in a libsph store plus its task list and buffers."""

    def __init__(self, fields: dict, layout="aos", seed: int = 0,
                 box=(1.0, 1.0, 1.0), bundle_max_slots: int = 0,
                 ncell=(0, 0, 0), params: sph.Params | None = None,
                 device: str = "cuda", share: "Offload | None" = None,
                 plan: str = "grid", leaf_max: int = 64):
        """``share``: reuse another Offload's task list, permutation and
        buffers (same particles, different store layout).  ``plan="tree"``:
        no uniform grid or per-task list; the particles are ordered by the
        octree-leaf plan of the batched pipeline (clustered sets), and only
        the batched calls are available."""
        if plan not in ("grid", "tree"):
            raise ValueError("plan must be 'grid' or 'tree'")
        self.plan = plan if share is None else share.plan
        self.leaf_max = leaf_max if share is None else share.leaf_max
        self.device = torch.device(device)
        self.layout = sph.LAYOUTS[layout] if isinstance(layout, str) else int(layout)
        self.seed = seed
        self.params = params or sph.params()
        x = np.ascontiguousarray(fields["x"], np.float64)
        self.n = n = x.shape[0]
        self.box = tuple(float(b) for b in box)
        self.owner = share is None
        if share is None and self.plan == "tree":
            self._x = x
            self._h = np.ascontiguousarray(fields["h"], np.float32)
            self.perm = np.empty(n, np.int64)
            self.tasks = None
            self.bplan = sph.sph_batch_build_tree(
                n, x.ctypes.data, self._h.ctypes.data, self.box, self.params.kernel_gamma,
                leaf_max, 0, 128, self.perm.ctypes.data)
            self._batch_buffers()
            self.info = dict(sph.sph_batch_plan_info(self.bplan))
            self.info.update(slots=None, nbundles=None)
            self.d_perm = torch.from_numpy(self.perm).to(self.device)
            self.buf_in = self.buf_out = None
        elif share is None:
            h = np.ascontiguousarray(fields["h"], np.float32)
            gp = sph.grid_params(box, self.params.kernel_gamma, ncell, bundle_max_slots)
            self.perm = np.empty(n, np.int64)
            self.tasks = sph.sph_tasks_build(n, x.ctypes.data, h.ctypes.data, gp,
                                             self.perm.ctypes.data)
            sph.sph_tasks_upload(self.tasks)
            self.info = sph.sph_tasks_info(self.tasks)
            self.d_perm = torch.from_numpy(self.perm).to(self.device)
            nin = max(sph.sph_buffer_bytes(self.tasks, l, 0) for l in range(3))
            nout = max(sph.sph_buffer_bytes(self.tasks, l, 1) for l in range(3))
            self.buf_in = torch.empty(max(nin, 256), dtype=torch.uint8, device=self.device)
            self.buf_out = torch.empty(max(nout, 256), dtype=torch.uint8, device=self.device)
        else:
            self.perm, self.tasks, self.info = share.perm, share.tasks, share.info
            self.d_perm, self.buf_in, self.buf_out = share.d_perm, share.buf_in, share.buf_out
            if self.plan == "tree":
                self._x, self._h = share._x, share._h
                self.use_batch_of(share)
        self.nbytes = sph.sph_store_bytes(n, self.layout, seed)
        self.mem = torch.empty(max(self.nbytes, 256), dtype=torch.uint8, device=self.device)
        self.store = sph.sph_store_create(n, self.layout, seed, self.mem.data_ptr(),
                                          self.nbytes)
        self.import_fields(fields)

    # -- plumbing --------------------------------------------------------
    @property
    def stream(self) -> int:
        return torch.cuda.current_stream(self.device).cuda_stream

    def nbundles(self) -> int:
        return self.info["nbundles"]

    def import_fields(self, fields: dict, names=INPUTS) -> None:
        dev = {}
        for name in names:
            if name not in fields:
                continue
            dt, k = field_spec(name)
            arr = np.ascontiguousarray(fields[name], dt)
            dev[name] = torch.from_numpy(arr).to(self.device)
        sph.sph_store_import(self.store, fields_struct(dev), self.d_perm.data_ptr(),
                             self.stream)
        torch.cuda.synchronize(self.device)

    def import_device(self, tensors: dict) -> None:
        """Copy device tensors (original particle order, contiguous, the
        field's dtype) into the store on the offload's stream."""
        sph.sph_store_import(self.store, fields_struct(tensors), self.d_perm.data_ptr(),
                             self.stream)

    def export_device(self, names) -> dict:
        """Store fields as device tensors in original particle order (enqueued
        on the offload's stream; no host synchronisation)."""
        dev = self.device_fields(names)
        sph.sph_store_export(self.store, fields_struct(dev), self.d_perm.data_ptr(),
                             self.stream)
        return dev

    def adjoint(self, abar, ebar, recompute_lists: bool = True):
        """Gradient of sum |a|^2 + sum (du/dt)^2 through the last list step,
        for upstream adjoints abar (n, 3) and ebar (n,) on the device; returns
        device tensors (dL/dx (n, 3) FP64, dL/dm (n,), dL/du (n,)).

        The pair lists are recomputed from the store's positions and
        supports before the backward (one list build), so the backward does
        not depend on lists kept from the forward; the pool they are built
        in is the Offload's own list buffer, reused rather than duplicated.
        recompute_lists=False takes the lists the last step left instead."""
        need = sph.sph_batch_adjoint_bytes(self.bplan)
        if need == 0:
            raise sph.SphError(6, "the adjoint needs a plan of one bundle")
        if recompute_lists or getattr(self, "blist", None) is None:
            self.list_build()
        if getattr(self, "adj_scratch", None) is None or self.adj_scratch.numel() < need:
            self.adj_scratch = torch.empty(need, dtype=torch.uint8, device=self.device)
        abar = abar.to(self.device, torch.float32).contiguous()
        ebar = ebar.to(self.device, torch.float32).contiguous()
        gx = torch.empty((self.n, 3), dtype=torch.float64, device=self.device)
        gm = torch.empty(self.n, dtype=torch.float32, device=self.device)
        gu = torch.empty(self.n, dtype=torch.float32, device=self.device)
        sph.sph_batch_adjoint(self.store, self.bplan, self.bbuf_in.data_ptr(),
                              self.blist.data_ptr(), self.blist_bytes,
                              self.adj_scratch.data_ptr(), self.adj_scratch.numel(),
                              self.d_perm.data_ptr(), abar.data_ptr(), ebar.data_ptr(),
                              gx.data_ptr(), gm.data_ptr(), gu.data_ptr(), self.params,
                              self.stream)
        return gx, gm, gu

    def device_fields(self, names) -> dict:
        out = {}
        for name in names:
            dt, k = field_spec(name)
            shape = (self.n, k) if k > 1 else (self.n,)
            out[name] = torch.empty(shape, dtype=_TORCH_DT[dt], device=self.device)
        return out

    def export(self, names=OUTPUTS) -> dict:
        dev = self.device_fields(names)
        sph.sph_store_export(self.store, fields_struct(dev), self.d_perm.data_ptr(),
                             self.stream)
        sph.sph_sync(self.stream)
        return {k: v.cpu().numpy() for k, v in dev.items()}

    def store_bytes(self) -> np.ndarray:
        torch.cuda.synchronize(self.device)
        return self.mem[: self.nbytes].cpu().numpy()

    # -- the offload cycle ----------------------------------------------
    def loop(self, loop: int) -> None:
        sph.sph_offload_loop(self.store, self.tasks, loop, self.buf_in.data_ptr(),
                             self.buf_out.data_ptr(), self.params, self.stream)

    def step(self) -> None:
        """density -> ghost -> gradient -> force over all bundles."""
        for loop in (sph.SPH_DENSITY, sph.SPH_GRADIENT, sph.SPH_FORCE):
            self.loop(loop)

    def pack(self, loop: int, bundle: int) -> None:
        sph.sph_pack(self.store, self.tasks, loop, bundle, self.buf_in.data_ptr(),
                     self.stream)

    def interact(self, loop: int, bundle: int) -> None:
        fn = (sph.sph_density, sph.sph_gradient, sph.sph_force)[loop]
        fn(self.tasks, bundle, self.buf_in.data_ptr(), self.buf_out.data_ptr(),
           self.params, self.stream)

    def unpack(self, loop: int, bundle: int) -> None:
        sph.sph_unpack(self.store, self.tasks, loop, bundle, self.buf_out.data_ptr(),
                       self.stream)

    def count_pairs(self, loop: int) -> int:
        """Pair interactions of `loop` (packs each bundle into buf_in)."""
        if self.plan == "tree":
            return self.count_pairs_fp64(loop)
        cnt = torch.zeros(1, dtype=torch.int64, device=self.device)
        for b in range(self.nbundles()):
            self.pack(loop, b)
            sph.sph_count_pairs(self.tasks, loop, b, self.buf_in.data_ptr(), self.params,
                                cnt.data_ptr(), self.stream)
        sph.sph_sync(self.stream)
        return int(cnt.item())

    def bundle_slots(self, bundle: int) -> int:
        bs = self.bundle_starts()
        return int(self.slot_counts()[bs[bundle]:bs[bundle + 1]].sum())

    def task_list(self):
        nt = self.info["ntasks"]
        ncell = self.info["ncell_x"] * self.info["ncell_y"] * self.info["ncell_z"]
        ci = np.empty(nt, np.int32)
        cj = np.empty(nt, np.int32)
        sh = np.empty((nt, 3), np.int8)
        cs = np.empty(ncell + 1, np.int64)
        bs = np.empty(self.info["nbundles"] + 1, np.int64)
        sph.sph_tasks_get(self.tasks, ci.ctypes.data, cj.ctypes.data, sh.ctypes.data,
                          cs.ctypes.data, bs.ctypes.data)
        return ci, cj, sh, cs, bs

    def bundle_starts(self):
        return self.task_list()[4]

    def slot_counts(self):
        ci, cj, sh, cs, bs = self.task_list()
        cnt = np.diff(cs)
        return cnt[ci] + np.where(cj >= 0, cnt[np.maximum(cj, 0)], 0)

    # -- batched (cell-dedup) cycle --------------------------------------
    def batch(self, max_target_cells: int = 0, threads: int = 128,
              leaf_max: int | None = None) -> None:
        """Build the batched plan for this particle set and its buffers
        (``leaf_max``: tree plan only; the leaves' Morton order, and so the
        store order, does not depend on it)."""
        self.close_batch()
        if leaf_max is not None:
            if self.plan != "tree":
                raise ValueError("leaf_max applies to the tree plan only")
            self.leaf_max = leaf_max
        if self.plan == "tree":
            perm = np.empty(self.n, np.int64)
            self.bplan = sph.sph_batch_build_tree(
                self.n, self._x.ctypes.data, self._h.ctypes.data, self.box,
                self.params.kernel_gamma, self.leaf_max, max_target_cells, threads,
                perm.ctypes.data)
            if not np.array_equal(perm, self.perm):
                raise RuntimeError("tree plan order changed for the same particles")
        else:
            self.bplan = sph.sph_batch_build(self.tasks, max_target_cells, threads)
        self.bshared = False
        self._batch_buffers()

    def _batch_buffers(self) -> None:
        self.binfo = sph.sph_batch_info(self.bplan)
        self.binfo.update(sph.sph_batch_plan_info(self.bplan))
        nin = max(sph.sph_batch_buffer_bytes(self.bplan, l, 0) for l in range(3))
        nout = max(sph.sph_batch_buffer_bytes(self.bplan, l, 1) for l in range(3))
        self.bbuf_in = torch.empty(max(nin, 256), dtype=torch.uint8, device=self.device)
        self.bbuf_out = torch.empty(max(nout, 256), dtype=torch.uint8, device=self.device)

    def use_batch_of(self, other: "Offload") -> None:
        """Share another Offload's batched plan and buffers."""
        self.bplan, self.binfo = other.bplan, other.binfo
        self.bbuf_in, self.bbuf_out = other.bbuf_in, other.bbuf_out
        self.blist = getattr(other, "blist", None)
        self.blist_bytes = getattr(other, "blist_bytes", 0)
        self.bshared = True

    def batch_loop(self, loop: int) -> None:
        sph.sph_batch_offload_loop(self.store, self.bplan, loop, self.bbuf_in.data_ptr(),
                                   self.bbuf_out.data_ptr(), self.params, self.stream)

    def batch_step(self) -> None:
        for loop in (sph.SPH_DENSITY, sph.SPH_GRADIENT, sph.SPH_FORCE):
            self.batch_loop(loop)

    def count_pairs_fp64(self, loop: int) -> int:
        """Pair interactions of `loop` over the batched plan, decided in FP64."""
        self._fp64_buffers()
        cnt = torch.zeros(1, dtype=torch.int64, device=self.device)
        sph.sph_batch_count_pairs(self.store, self.bplan, loop, self.f64_in.data_ptr(),
                                  self.params, cnt.data_ptr(), self.stream)
        return int(cnt.item())

    def _fp64_buffers(self) -> None:
        if getattr(self, "f64_in", None) is None:
            nin = sph.sph_batch_buffer_bytes_fp64(self.bplan, 0)
            nout = sph.sph_batch_buffer_bytes_fp64(self.bplan, 1)
            self.f64_in = torch.empty(max(nin, 256), dtype=torch.uint8, device=self.device)
            self.f64_out = torch.empty(max(nout, 256), dtype=torch.uint8, device=self.device)

    def fp64_step(self) -> None:
        """The batched step with every arithmetic step in FP64."""
        self._fp64_buffers()
        for loop in (sph.SPH_DENSITY, sph.SPH_GRADIENT, sph.SPH_FORCE):
            sph.sph_batch_offload_loop_fp64(self.store, self.bplan, loop, self.f64_in.data_ptr(),
                                            self.f64_out.data_ptr(), self.params, self.stream)

    # -- neighbour-list variant ---------------------------------------------
    def _alloc_list(self, chunks: int) -> None:
        self.blist = None
        torch.cuda.empty_cache()
        self.blist_bytes = sph.sph_batch_list_bytes(self.bplan, chunks)
        self.blist = torch.empty(self.blist_bytes, dtype=torch.uint8, device=self.device)

    def list_build(self) -> None:
        """Build the per-step neighbour lists (sized on first use: one
        synchronous status read, the pool grown if it ran out)."""
        if getattr(self, "blist", None) is None:
            self._alloc_list(int(1.25 * self.binfo["items"]) + 16)
            for _ in range(3):
                sph.sph_batch_list_build(self.store, self.bplan, self.bbuf_in.data_ptr(),
                                         self.blist.data_ptr(), self.blist_bytes, self.params,
                                         self.stream)
                need, overflow = sph.sph_batch_list_status(self.blist.data_ptr())
                if not overflow:
                    break
                try:
                    sph.sph_sync(self.stream)      # clears the latched pool error
                except sph.SphError:
                    pass
                if overflow == 2:
                    raise sph.SphError(6, "a particle has more neighbours than one list chain "
                                       "holds (16384)")
                self._alloc_list(int(1.05 * need) + 16)
            return
        sph.sph_batch_list_build(self.store, self.bplan, self.bbuf_in.data_ptr(),
                                 self.blist.data_ptr(), self.blist_bytes, self.params,
                                 self.stream)

    def list_loop(self, loop: int) -> None:
        sph.sph_batch_offload_loop_list(self.store, self.bplan, loop, self.bbuf_in.data_ptr(),
                                        self.bbuf_out.data_ptr(), self.blist.data_ptr(),
                                        self.blist_bytes, self.params, self.stream)

    def list_step(self) -> None:
        """Lists, then density -> ghost -> gradient -> force over them, in one
        library call (the density pack serves the list build too).  The first
        call sizes the list pool with a separate build.  Later steps only
        enqueue: if moved particles need more list entries than the pool
        holds, the step's loops skip all pairs and the next sph_sync raises
        SPH_ENOMEM; resize() then regrows the pool for the next step."""
        if getattr(self, "blist", None) is None:
            self.list_build()
        sph.sph_batch_offload_step_list(self.store, self.bplan, self.bbuf_in.data_ptr(),
                                        self.bbuf_out.data_ptr(), self.blist.data_ptr(),
                                        self.blist_bytes, self.params, self.stream)

    def list_step_x64(self) -> None:
        """The list step with FP64 pair separations (precision study)."""
        if getattr(self, "blist", None) is None:
            self.list_build()
        need = sph.sph_batch_x64_bytes(self.bplan)
        if getattr(self, "x64", None) is None or self.x64.numel() < need:
            self.x64 = torch.empty(max(need, 256), dtype=torch.uint8, device=self.device)
        sph.sph_batch_offload_step_list_x64(self.store, self.bplan, self.bbuf_in.data_ptr(),
                                            self.bbuf_out.data_ptr(), self.blist.data_ptr(),
                                            self.blist_bytes, self.x64.data_ptr(),
                                            self.x64.numel(), self.params, self.stream)

    def resize(self) -> None:
        """Size the list pool again for the current positions (one
        synchronous build and status read)."""
        self.blist = None
        self.list_build()

    def close_batch(self) -> None:
        self.f64_in = self.f64_out = None
        self.x64 = None
        self.blist = None
        if getattr(self, "bplan", None) is not None:
            if not getattr(self, "bshared", False):
                sph.sph_batch_destroy(self.bplan)
            self.bplan = None

    def close(self) -> None:
        self.close_batch()
        if getattr(self, "store", None) is not None:
            sph.sph_store_destroy(self.store)
            self.store = None
        if getattr(self, "tasks", None) is not None:
            if self.owner:
                sph.sph_tasks_destroy(self.tasks)
            self.tasks = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def aligned_host(nbytes: int, pinned: bool = False):
    """A 256-byte aligned host byte buffer: (array view, owner).  Pinned
    memory comes from torch (needs a CUDA device); otherwise numpy."""
    nbytes = max(int(nbytes), 256)
    if pinned:
        t = torch.empty(nbytes + 256, dtype=torch.uint8).pin_memory()
        off = (-t.data_ptr()) % 256
        return t[off:off + nbytes].numpy(), t
    a = np.empty(nbytes + 256, np.uint8)
    off = (-a.ctypes.data) % 256
    return a[off:off + nbytes], a


def host_fields_struct(arrays: dict) -> sph.Fields:
    F = sph.Fields()
    for name, a in arrays.items():
        if a is None:
            continue
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("field %s must be C-contiguous" % name)
        setattr(F, name, a.ctypes.data)
    return F


def pinned_fields(n: int, names) -> dict:
    """Page-locked host tensors for the named fields of n particles."""
    out = {}
    for name in names:
        dt, k = field_spec(name)
        shape = (n, k) if k > 1 else (n,)
        out[name] = torch.empty(shape, dtype=_TORCH_DT[dt]).pin_memory()
    return out


class StreamingSteps:
    """End-to-end steps from pinned host inputs to pinned host results,
    entirely through the library's host I/O handle (sph_hostio_*): each step
    copies its inputs host -> device and imports them, runs `step_fn` (library
    calls on the offload's stream), exports its results and copies them
    device -> host.  The library double-buffers the device staging and issues
    the copies on two copy streams, so step k+1's inputs and step k-1's
    results travel while step k computes."""

    def __init__(self, off: "Offload", step_fn, names_in=INPUTS, names_out=OUTPUTS):
        self.off = off
        self.step_fn = step_fn
        self.names_in, self.names_out = tuple(names_in), tuple(names_out)
        sel_in, sel_out = sph.Fields(), sph.Fields()
        for name in self.names_in:
            setattr(sel_in, name, 1)
        for name in self.names_out:
            setattr(sel_out, name, 1)
        nbytes = sph.sph_hostio_bytes(off.n, sel_in, sel_out)
        self.staging = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=off.device)
        self.s_in = torch.cuda.Stream(off.device)
        self.s_out = torch.cuda.Stream(off.device)
        self.io = sph.sph_hostio_create(off.store, off.d_perm.data_ptr(), sel_in, sel_out,
                                        self.staging.data_ptr(), nbytes,
                                        self.s_in.cuda_stream, self.s_out.cuda_stream)

    def pinned_in(self) -> dict:
        return pinned_fields(self.off.n, self.names_in)

    def pinned_out(self) -> dict:
        return pinned_fields(self.off.n, self.names_out)

    def bytes_per_step(self):
        info = sph.sph_hostio_info(self.io)
        return info["h2d_bytes_per_step"], info["d2h_bytes_per_step"]

    def step(self, pin_in: dict, pin_out: dict) -> None:
        """Enqueue one step: H2D of pin_in, the step, D2H into pin_out (all
        arrays page-locked, original particle order)."""
        sph.sph_hostio_begin(self.io, fields_struct(pin_in), self.off.stream)
        self.step_fn()
        sph.sph_hostio_end(self.io, fields_struct(pin_out), self.off.stream)

    def drain(self) -> None:
        """The offload's stream waits for the last step's results."""
        sph.sph_hostio_drain(self.io, self.off.stream)

    def close(self) -> None:
        if getattr(self, "io", None) is not None:
            sph.sph_hostio_destroy(self.io)
            self.io = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class HostOffload:
    """A particle set in a host-memory store (the paper's host side) with the
    host-staged double-buffered cycle.  Without a GPU only the host calls
    (import/export, pack, unpack, init, ghost) are usable."""

    def __init__(self, fields: dict, layout="aos", seed: int = 0, box=(1.0, 1.0, 1.0),
                 bundle_max_slots: int = 0, ncell=(0, 0, 0),
                 params: sph.Params | None = None, gpu: bool = True, nthreads: int = 0,
                 plan: str = "grid", leaf_max: int = 128, max_target_cells: int = 0,
                 threads: int = 128):
        """plan "grid": the per-task cycle's cells and tasks (and, through
        batch_step, the batched cycle on them); plan "tree": octree leaves
        for clustered sets, batched cycle only (needs the GPU)."""
        self.layout = sph.LAYOUTS[layout] if isinstance(layout, str) else int(layout)
        self.params = params or sph.params()
        self.nthreads = nthreads
        self.gpu = gpu
        self.plan = plan
        self.seed, self.box, self.leaf_max = seed, tuple(float(b) for b in box), leaf_max
        x = np.ascontiguousarray(fields["x"], np.float64)
        h = np.ascontiguousarray(fields["h"], np.float32)
        self.n = n = x.shape[0]
        self.perm = np.empty(n, np.int64)
        self.tasks = self.bplan = None
        if plan == "tree":
            if not gpu:
                raise ValueError("the tree plan lives on the device: gpu=True")
            self.bplan = sph.sph_batch_build_tree(n, x.ctypes.data, h.ctypes.data, box,
                                                  self.params.kernel_gamma, leaf_max,
                                                  max_target_cells, threads,
                                                  self.perm.ctypes.data)
            self.info = dict(sph.sph_batch_info(self.bplan))
        else:
            gp = sph.grid_params(box, self.params.kernel_gamma, ncell, bundle_max_slots)
            self.tasks = sph.sph_tasks_build(n, x.ctypes.data, h.ctypes.data, gp,
                                             self.perm.ctypes.data)
            self.info = sph.sph_tasks_info(self.tasks)
        self.nbytes = sph.sph_store_bytes(n, self.layout, seed)
        self.mem, self._mem_owner = aligned_host(self.nbytes, pinned=gpu)
        self.store = sph.sph_store_create_host(n, self.layout, seed, self.mem.ctypes.data,
                                               self.nbytes)
        self.host_in = self.host_out = None
        if self.tasks is not None:
            nin = max(sph.sph_buffer_bytes(self.tasks, l, 0) for l in range(3))
            nout = max(sph.sph_buffer_bytes(self.tasks, l, 1) for l in range(3))
            self.nin, self.nout = nin, nout
            self.host_in = [aligned_host(nin, pinned=gpu) for _ in range(2)]
            self.host_out = [aligned_host(nout, pinned=gpu) for _ in range(2)]
        if gpu:
            self.streams = [torch.cuda.Stream() for _ in range(2)]
        if gpu and self.tasks is not None:
            sph.sph_tasks_upload(self.tasks)
            self.dev_in = [torch.empty(max(nin, 256), dtype=torch.uint8, device="cuda")
                           for _ in range(2)]
            self.dev_out = [torch.empty(max(nout, 256), dtype=torch.uint8, device="cuda")
                            for _ in range(2)]
        self.import_fields(fields)

    def batch(self, max_target_cells: int = 0, threads: int = 128) -> None:
        """Batched plan of the grid's cells (the tree plan is built already)."""
        if self.plan == "tree":
            return
        if self.bplan is not None:
            sph.sph_batch_destroy(self.bplan)
        self.bplan = sph.sph_batch_build(self.tasks, max_target_cells, threads)
        self.bbufs = None

    def batch_loop(self, loop: int) -> None:
        if self.bplan is None:
            self.batch()
        if getattr(self, "bbufs", None) is None:
            nin = max(sph.sph_batch_buffer_bytes(self.bplan, l, 0) for l in range(3))
            nout = max(sph.sph_batch_buffer_bytes(self.bplan, l, 1) for l in range(3))
            self.bbufs = (
                [aligned_host(nin, pinned=True) for _ in range(2)],
                [aligned_host(nout, pinned=True) for _ in range(2)],
                [torch.empty(max(nin, 256), dtype=torch.uint8, device="cuda") for _ in range(2)],
                [torch.empty(max(nout, 256), dtype=torch.uint8, device="cuda") for _ in range(2)])
        hin, hout, din, dout = self.bbufs
        sph.sph_batch_offload_loop_host(
            self.store, self.bplan, loop, [b[0].ctypes.data for b in hin],
            [b[0].ctypes.data for b in hout], [d.data_ptr() for d in din],
            [d.data_ptr() for d in dout], self.params, [s.cuda_stream for s in self.streams],
            self.nthreads)

    def batch_step(self) -> None:
        """The batched cycle from the host store (host-staged)."""
        for loop in (sph.SPH_DENSITY, sph.SPH_GRADIENT, sph.SPH_FORCE):
            self.batch_loop(loop)

    def import_fields(self, fields: dict, names=INPUTS) -> None:
        keep = {}
        for name in names:
            if name in fields:
                dt, k = field_spec(name)
                keep[name] = np.ascontiguousarray(fields[name], dt)
        sph.sph_store_import_host(self.store, host_fields_struct(keep), self.perm.ctypes.data,
                                  self.nthreads)

    def export(self, names=OUTPUTS) -> dict:
        out = {}
        for name in names:
            dt, k = field_spec(name)
            out[name] = np.empty((self.n, k) if k > 1 else (self.n,), dt)
        sph.sph_store_export_host(self.store, host_fields_struct(out), self.perm.ctypes.data,
                                  self.nthreads)
        return out

    def store_bytes(self) -> np.ndarray:
        return self.mem[: self.nbytes].copy()

    def loop(self, loop: int) -> None:
        sph.sph_offload_loop_host(
            self.store, self.tasks, loop, [b[0].ctypes.data for b in self.host_in],
            [b[0].ctypes.data for b in self.host_out], [d.data_ptr() for d in self.dev_in],
            [d.data_ptr() for d in self.dev_out], self.params,
            [s.cuda_stream for s in self.streams], self.nthreads)

    def step(self) -> None:
        for loop in (sph.SPH_DENSITY, sph.SPH_GRADIENT, sph.SPH_FORCE):
            self.loop(loop)

    def loop_stats(self, loop: int) -> dict:
        """One loop of the host-staged cycle with every stage timed
        (sph_offload_loop_host_stats)."""
        return sph.sph_offload_loop_host_stats(
            self.store, self.tasks, loop, [b[0].ctypes.data for b in self.host_in],
            [b[0].ctypes.data for b in self.host_out], [d.data_ptr() for d in self.dev_in],
            [d.data_ptr() for d in self.dev_out], self.params,
            [s.cuda_stream for s in self.streams], self.nthreads)

    def step_stats(self) -> list:
        """A step with every stage timed: the stats of each loop."""
        return [self.loop_stats(loop)
                for loop in (sph.SPH_DENSITY, sph.SPH_GRADIENT, sph.SPH_FORCE)]

    def task_list(self):
        nt = self.info["ntasks"]
        ncell = self.info["ncell_x"] * self.info["ncell_y"] * self.info["ncell_z"]
        ci = np.empty(nt, np.int32)
        cj = np.empty(nt, np.int32)
        sh = np.empty((nt, 3), np.int8)
        cs = np.empty(ncell + 1, np.int64)
        bs = np.empty(self.info["nbundles"] + 1, np.int64)
        sph.sph_tasks_get(self.tasks, ci.ctypes.data, cj.ctypes.data, sh.ctypes.data,
                          cs.ctypes.data, bs.ctypes.data)
        return ci, cj, sh, cs, bs

    def close(self) -> None:
        if getattr(self, "store", None) is not None:
            sph.sph_store_destroy(self.store)
            self.store = None
        if getattr(self, "tasks", None) is not None:
            sph.sph_tasks_destroy(self.tasks)
            self.tasks = None
        if getattr(self, "bplan", None) is not None:
            sph.sph_batch_destroy(self.bplan)
            self.bplan = None
        self.bbufs = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
