"""Autotuner choices kept across processes.

libpf keeps the tile size that ``pf_autotune`` picks for a (device, kind, size
class) only for the life of the process.  This module stores those picks in a
JSON file keyed by the device model, and loads them back in a later process
through ``pf_set_min_tile``, so that a tuned tiling is measured once per GPU
model instead of once per run.  Host bookkeeping only: the timing is the
library's own (``pf_autotune``), and nothing here runs on the device.

File layout::

    {"version": 1,
     "devices": {"<device key>": {"systematic": {"20": 4096, ...},
                                  "stratified": {...}, "multinomial": {...}}}}

A size class is ceil(log2 P) (P = 1 is class 0), the granularity at which the
library keeps its choices; a choice stored for class c is set again through
``pf_set_min_tile(kind, 2**c, tile)``.  The device key names the model, its SM
count and compute capability, so a file made on one GPU model is never
applied to another.
"""
from __future__ import annotations

import json
import os
import tempfile

from . import pf

VERSION = 1
KIND_NAMES = {pf.PF_MULTINOMIAL: "multinomial", pf.PF_STRATIFIED: "stratified", pf.PF_SYSTEMATIC: "systematic"}
N_CLASSES = 32  # the library keeps size classes 0..31


def size_class(P: int) -> int:
    """ceil(log2 P), capped at N_CLASSES - 1: the library's size class of P."""
    if P < 1:
        raise ValueError("P must be >= 1")
    return min((int(P) - 1).bit_length(), N_CLASSES - 1)


def device_key(device=None) -> str:
    """'<name>|<SMs> SMs|sm_<major><minor>' of a CUDA device (torch's current one by default)."""
    import torch
    p = torch.cuda.get_device_properties(torch.cuda.current_device() if device is None else device)
    return f"{p.name}|{p.multi_processor_count} SMs|sm_{p.major}{p.minor}"


def read(path: str) -> dict:
    """The file's contents ({"version", "devices"}); an empty table when the file does not exist.
    Raises ValueError for a file of another layout."""
    if not os.path.exists(path):
        return {"version": VERSION, "devices": {}}
    with open(path) as f:
        data = json.load(f)
    if not isinstance(data, dict) or data.get("version") != VERSION or not isinstance(data.get("devices"), dict):
        raise ValueError(f"{path}: not a version-{VERSION} tile-size file")
    for key, kinds in data["devices"].items():
        if not isinstance(kinds, dict):
            raise ValueError(f"{path}: entry {key!r} is not a table of kinds")
        for kind, classes in kinds.items():
            if kind not in KIND_NAMES.values() or not isinstance(classes, dict):
                raise ValueError(f"{path}: unknown kind {kind!r} for {key!r}")
            for c, tile in classes.items():
                if not (c.isdigit() and int(c) < N_CLASSES and isinstance(tile, int) and tile >= 0):
                    raise ValueError(f"{path}: bad entry {kind}[{c!r}] = {tile!r} for {key!r}")
    return data


def record(path: str, key: str, kind: int, P: int, min_tile: int) -> None:
    """Store one choice for (key, kind, size class of P), replacing the file atomically."""
    if kind not in KIND_NAMES:
        raise ValueError(f"kind {kind}: only the multinomial, stratified and systematic calls are tiled")
    data = read(path)
    classes = data["devices"].setdefault(key, {}).setdefault(KIND_NAMES[kind], {})
    classes[str(size_class(P))] = int(min_tile)
    d = os.path.dirname(os.path.abspath(path))
    fd, tmp = tempfile.mkstemp(prefix=".tiles-", dir=d)
    try:
        with os.fdopen(fd, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except BaseException:
        os.unlink(tmp)
        raise


def tune_and_record(path: str, kind: int, logw, P: int, ancestors, reps: int = 20, stream=None, key=None):
    """Run pf_autotune for (kind, P) on the caller's log-weights and store its pick under
    this device's key.  Returns (min_tile, microseconds per call) as pf_autotune does."""
    tile, us = pf.pf_autotune(kind, logw, P, ancestors, reps=reps, stream=stream)
    record(path, device_key() if key is None else key, kind, P, tile)
    return tile, us


def load(path: str, key=None) -> int:
    """Set every choice the file holds for this device (pf_set_min_tile) and return how
    many were set; a missing file or another device's entries set nothing."""
    data = read(path)
    kinds = data["devices"].get(device_key() if key is None else key, {})
    by_name = {v: k for k, v in KIND_NAMES.items()}
    n = 0
    for name, classes in kinds.items():
        for c, tile in classes.items():
            pf.pf_set_min_tile(by_name[name], 1 << int(c), tile)
            n += 1
    return n
