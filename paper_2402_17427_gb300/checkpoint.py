"""Checkpoint and resume of one cell's training state.

A cell's state is its Gaussians as structure-of-arrays (means [n,3], log-scales [n,3], quaternions
[n,4], opacity logits [n], SH coefficients [n,K,3]), the Adam moments and step count of each
array, the densification statistics, and optionally the appearance CNN's parameters and the
per-view embeddings (paper Sec. 4.2), with the iteration number.  Cells train independently
(Sec. 4.1), so each cell is one file.

File format (little-endian, written by this module only):
    8 bytes    magic b"VGCKPT01"
    8 bytes    u64 length J of the header
    J bytes    UTF-8 JSON header: {"meta": {...}, "arrays": [{"name", "dtype", "shape", "offset",
               "nbytes", "sha256"}, ...]}
    ...        each array's raw bytes (C order) at header end + offset, 64-byte aligned
A file is written to a temporary name in the same directory and renamed over the target only
after it is complete and flushed, so a crash mid-write leaves the previous checkpoint intact.
Loading verifies every array's SHA-256 and raises ``CheckpointError`` on any mismatch,
truncation or unknown format.
"""
from __future__ import annotations

import hashlib
import json
import os
import struct
import tempfile

import numpy as np
import torch

MAGIC = b"VGCKPT01"
_ALIGN = 64
PARAM_NAMES = ("means", "log_scales", "quats", "opacity_logits", "sh")


class CheckpointError(RuntimeError):
    pass


def _host(t: torch.Tensor) -> np.ndarray:
    return t.detach().contiguous().cpu().numpy()


def save(path: str, params, degree: int, iteration: int = 0, adam=None, stats=None, appearance=None,
         meta: dict | None = None) -> None:
    """Writes the state to `path` atomically.  params: the five parameter tensors (any device);
    adam: an ``optim.Adam`` (moments and step count); stats: an ``optim.DensifyStats``;
    appearance: an ``appearance.AppearanceModel``."""
    arrays: list[tuple[str, np.ndarray]] = []
    for name, t in zip(PARAM_NAMES, params):
        arrays.append((name, _host(t)))
    head = {"degree": int(degree), "iteration": int(iteration), "n": int(params[0].shape[0])}
    if adam is not None:
        for name, m, v in zip(PARAM_NAMES, adam.m, adam.v):
            arrays.append(("adam_m/" + name, _host(m)))
            arrays.append(("adam_v/" + name, _host(v)))
        head["adam_step"] = int(adam.t)
    if stats is not None:
        arrays.append(("densify/accum", _host(stats.accum)))
        arrays.append(("densify/count", _host(stats.count)))
    if appearance is not None:
        arrays.append(("appearance/params", _host(appearance.params)))
        arrays.append(("appearance/embeddings", _host(appearance.embeddings)))
    head["user"] = dict(meta or {})
    index, off = [], 0
    for name, a in arrays:
        off = (off + _ALIGN - 1) // _ALIGN * _ALIGN
        index.append({"name": name, "dtype": a.dtype.str, "shape": list(a.shape), "offset": off,
                      "nbytes": int(a.nbytes), "sha256": hashlib.sha256(a.tobytes()).hexdigest()})
        off += a.nbytes
    header = json.dumps({"meta": head, "arrays": index}).encode()
    d = os.path.dirname(os.path.abspath(path))
    fd, tmp = tempfile.mkstemp(prefix=".vgckpt-", dir=d)
    try:
        with os.fdopen(fd, "wb") as f:
            f.write(MAGIC)
            f.write(struct.pack("<Q", len(header)))
            f.write(header)
            base = f.tell()
            for (name, a), e in zip(arrays, index):
                f.seek(base + e["offset"])
                f.write(a.tobytes())
            f.flush()
            os.fsync(f.fileno())
        os.replace(tmp, path)
    except BaseException:
        if os.path.exists(tmp):
            os.unlink(tmp)
        raise


def read(path: str) -> tuple[dict, dict[str, np.ndarray]]:
    """(meta, {name: host array}) with every checksum verified."""
    with open(path, "rb") as f:
        if f.read(8) != MAGIC:
            raise CheckpointError(f"{path}: not a checkpoint of this format")
        raw = f.read(8)
        if len(raw) != 8:
            raise CheckpointError(f"{path}: truncated header")
        (hl,) = struct.unpack("<Q", raw)
        try:
            header = json.loads(f.read(hl).decode())
        except (UnicodeDecodeError, json.JSONDecodeError) as e:
            raise CheckpointError(f"{path}: corrupt header") from e
        base = 16 + hl
        out = {}
        for e in header["arrays"]:
            f.seek(base + e["offset"])
            buf = f.read(e["nbytes"])
            if len(buf) != e["nbytes"]:
                raise CheckpointError(f"{path}: array {e['name']} truncated")
            if hashlib.sha256(buf).hexdigest() != e["sha256"]:
                raise CheckpointError(f"{path}: array {e['name']} fails its checksum")
            out[e["name"]] = np.frombuffer(buf, dtype=np.dtype(e["dtype"])).reshape(e["shape"]).copy()
    return header["meta"], out


def load(path: str, device="cuda", adam=None, stats=None, appearance=None):
    """Restores a state written by ``save``.  Returns (params, degree, iteration, meta); when given,
    `adam`, `stats` and `appearance` are filled in place from the file (each must have been
    saved)."""
    meta, arr = read(path)
    dev = torch.device(device)
    params = tuple(torch.from_numpy(arr[name]).to(dev) for name in PARAM_NAMES)
    if adam is not None:
        if "adam_step" not in meta:
            raise CheckpointError(f"{path}: holds no optimiser state")
        adam.m = tuple(torch.from_numpy(arr["adam_m/" + name]).to(dev) for name in PARAM_NAMES)
        adam.v = tuple(torch.from_numpy(arr["adam_v/" + name]).to(dev) for name in PARAM_NAMES)
        adam.t = int(meta["adam_step"])
    if stats is not None:
        if "densify/accum" not in arr:
            raise CheckpointError(f"{path}: holds no densification statistics")
        stats.accum = torch.from_numpy(arr["densify/accum"]).to(dev)
        stats.count = torch.from_numpy(arr["densify/count"]).to(dev)
    if appearance is not None:
        if "appearance/params" not in arr:
            raise CheckpointError(f"{path}: holds no appearance model")
        appearance.params = torch.from_numpy(arr["appearance/params"]).to(dev)
        appearance.embeddings = torch.from_numpy(arr["appearance/embeddings"]).to(dev)
    return params, int(meta["degree"]), int(meta["iteration"]), meta.get("user", {})
