"""Checkpoint and resume of a particle set.

A checkpoint holds every field of the particle store in the original particle
order, and what rebuilds the offload around it: the layout, its seed, the box,
the plan and the physics parameters.  Resuming imports the fields into a new
store, in the same or another layout, so the next step gives the results the
uninterrupted run would have given (bit for bit in the same layout).

File format (little-endian):
    b"SPHCKPT1\\n"
    8-byte unsigned header length L
    L bytes of JSON: {"meta": {...}, "fields": [{"name", "dtype", "shape",
                      "offset", "nbytes", "crc32"}, ...]}
    the raw arrays, each at its offset from the start of the data section,
    aligned to 64 bytes.
The readers check the magic, the sizes and each array's CRC-32 and raise
``ValueError`` on any mismatch.
"""
from __future__ import annotations

import json
import struct
import zlib

import numpy as np

from . import sph

MAGIC = b"SPHCKPT1\n"
ALIGN = 64


def write(path: str, meta: dict, arrays: dict) -> None:
    """Write ``arrays`` (name -> numpy array) and the JSON-able ``meta``."""
    fields, off = [], 0
    for name, a in arrays.items():
        a = np.ascontiguousarray(a)
        off = -(-off // ALIGN) * ALIGN
        fields.append({"name": name, "dtype": a.dtype.newbyteorder("<").str,
                       "shape": list(a.shape), "offset": off, "nbytes": a.nbytes,
                       "crc32": zlib.crc32(a.astype(a.dtype.newbyteorder("<")).tobytes())})
        off += a.nbytes
    head = json.dumps({"meta": meta, "fields": fields}).encode()
    with open(path, "wb") as fh:
        fh.write(MAGIC)
        fh.write(struct.pack("<Q", len(head)))
        fh.write(head)
        base = fh.tell()
        for f, a in zip(fields, arrays.values()):
            fh.seek(base + f["offset"])
            fh.write(np.ascontiguousarray(a, np.dtype(f["dtype"])).tobytes())


def read(path: str):
    """(meta, arrays) from a checkpoint file, every array checked."""
    with open(path, "rb") as fh:
        if fh.read(len(MAGIC)) != MAGIC:
            raise ValueError("%s: not a particle checkpoint" % path)
        raw = fh.read(8)
        if len(raw) != 8:
            raise ValueError("%s: truncated header" % path)
        (hl,) = struct.unpack("<Q", raw)
        head = fh.read(hl)
        if len(head) != hl:
            raise ValueError("%s: truncated header" % path)
        try:
            doc = json.loads(head)
        except json.JSONDecodeError as e:
            raise ValueError("%s: header is not JSON (%s)" % (path, e)) from None
        base = fh.tell()
        arrays = {}
        for f in doc["fields"]:
            fh.seek(base + f["offset"])
            buf = fh.read(f["nbytes"])
            if len(buf) != f["nbytes"]:
                raise ValueError("%s: field %s truncated" % (path, f["name"]))
            if zlib.crc32(buf) != f["crc32"]:
                raise ValueError("%s: field %s fails its CRC-32" % (path, f["name"]))
            dt = np.dtype(f["dtype"])
            arrays[f["name"]] = np.frombuffer(buf, dt).reshape(f["shape"]).astype(
                dt.newbyteorder("="))
    return doc["meta"], arrays


def save(off, path: str) -> None:
    """Checkpoint an ``Offload`` or a ``HostOffload``: all store fields after
    the work enqueued so far, and its layout, seed, box, plan and
    parameters."""
    p = off.params
    meta = {"n": off.n, "layout": off.layout, "seed": off.seed, "box": list(off.box),
            "plan": off.plan, "leaf_max": off.leaf_max,
            "params": {k: getattr(p, k) for k, _ in sph.Params._fields_ if k != "reserved"}}
    write(path, meta, off.export(sph.FIELD_NAMES))


def resume(path: str, layout=None, host: bool = False, **kwargs):
    """The checkpointed particles in a new ``Offload`` (``host``: a
    ``HostOffload``; ``kwargs`` go to its constructor), in the saved layout
    or in ``layout``.  The caller builds its batched plan as before."""
    from .pipeline import HostOffload, Offload
    meta, arrays = read(path)
    if len(arrays["x"]) != meta["n"]:
        raise ValueError("%s: %d particles in the header, %d stored"
                         % (path, meta["n"], len(arrays["x"])))
    cls = HostOffload if host else Offload
    off = cls(arrays, layout=meta["layout"] if layout is None else layout, seed=meta["seed"],
              box=tuple(meta["box"]), params=sph.params(**meta["params"]), plan=meta["plan"],
              leaf_max=meta["leaf_max"], **kwargs)
    off.import_fields(arrays, names=sph.FIELD_NAMES)
    return off
