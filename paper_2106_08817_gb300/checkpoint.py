"""Host files of an iterative registration, for stopping and resuming it.

A registration minimises the Eq. 4 cost of arXiv:2106.08817 over the initial
momentum p0 by gradient descent (the paper's optimiser, Sec. 3) or L-BFGS;
its state between iterations is the iterate p0, the iteration count, the
cost history and, for L-BFGS, the optimiser state image that the library
writes (meta_lbfgs_state_save: gradient, pair rings, rho, gamma, costs and
flags, with its own FNV-1a checksum).  This module only reads and writes
such files; paper_2106_08817_gb300.Registration saves and resumes through it.

Format: a NumPy .npz archive (no pickled objects) with the arrays
``format`` ("meta-registration"), ``version`` (1), ``meta`` (the settings as
a JSON string), ``p`` (float32), ``costs`` (float64 [iterations + 1, B]),
``images_sha256`` (of the I0 and J bytes, so that a file is not resumed on
other images) and, for L-BFGS, ``lbfgs_state`` (uint8).  Files are written
to a temporary name in the same directory and renamed over the target, so a
reader never sees half a file.
"""
from __future__ import annotations

import hashlib
import json
import os
from typing import Optional

import numpy as np

FORMAT = "meta-registration"
VERSION = 1
SETTINGS = ("optimizer", "ndim", "dims", "batch", "T", "sigma", "mu", "rho", "lam", "m", "h0",
            "ckpt", "p_update", "scheme", "iterations")

__all__ = ["FORMAT", "VERSION", "SETTINGS", "images_digest", "write", "read"]


def images_digest(I0: np.ndarray, J: np.ndarray) -> str:
    """SHA-256 of the float32 bytes of I0 then J (C order)."""
    h = hashlib.sha256()
    for a in (I0, J):
        h.update(np.ascontiguousarray(a, dtype=np.float32).tobytes())
    return h.hexdigest()


def write(path, settings: dict, p: np.ndarray, costs: np.ndarray, digest: str,
          lbfgs_state: Optional[bytes] = None) -> None:
    """Writes one registration state (atomically: temporary file, then rename)."""
    missing = [k for k in SETTINGS if k not in settings]
    if missing:
        raise ValueError("settings lack %s" % missing)
    if settings["optimizer"] not in ("gd", "lbfgs"):
        raise ValueError("optimizer must be 'gd' or 'lbfgs'")
    if (settings["optimizer"] == "lbfgs") != (lbfgs_state is not None):
        raise ValueError("an L-BFGS state goes with optimizer 'lbfgs' only")
    p = np.ascontiguousarray(p, dtype=np.float32)
    costs = np.ascontiguousarray(costs, dtype=np.float64)
    if costs.ndim != 2 or costs.shape[0] != settings["iterations"] + 1:
        raise ValueError("costs must be [iterations + 1, batch]")
    arrays = dict(format=np.array(FORMAT), version=np.array(VERSION, dtype=np.int64),
                  meta=np.array(json.dumps({k: settings[k] for k in SETTINGS}, sort_keys=True)),
                  p=p, costs=costs, images_sha256=np.array(digest))
    if lbfgs_state is not None:
        arrays["lbfgs_state"] = np.frombuffer(bytes(lbfgs_state), dtype=np.uint8)
    path = os.fspath(path)
    d = os.path.dirname(os.path.abspath(path))
    tmp = os.path.join(d, ".%s.tmp%d" % (os.path.basename(path), os.getpid()))
    try:
        with open(tmp, "wb") as f:
            np.savez(f, **arrays)
            f.flush()
            os.fsync(f.fileno())
        os.replace(tmp, path)
    finally:
        if os.path.exists(tmp):
            os.remove(tmp)


def read(path) -> dict:
    """Reads a file written by `write`: a dict with the settings, ``p``,
    ``costs``, ``images_sha256`` and ``lbfgs_state`` (bytes or None).  Raises
    ValueError for a file of another format or version, or whose arrays do
    not agree with its settings."""
    with np.load(os.fspath(path), allow_pickle=False) as z:
        names = set(z.files)
        if not {"format", "version", "meta", "p", "costs", "images_sha256"} <= names:
            raise ValueError("not a registration state file")
        if str(z["format"]) != FORMAT or int(z["version"]) != VERSION:
            raise ValueError("registration state format %s version %s is not %s version %d"
                             % (z["format"], z["version"], FORMAT, VERSION))
        out = json.loads(str(z["meta"]))
        out["p"] = np.array(z["p"], dtype=np.float32)
        out["costs"] = np.array(z["costs"], dtype=np.float64)
        out["images_sha256"] = str(z["images_sha256"])
        out["lbfgs_state"] = bytes(z["lbfgs_state"].tobytes()) if "lbfgs_state" in names else None
    if set(SETTINGS) - set(out):
        raise ValueError("registration state settings are incomplete")
    shape = (out["batch"],) + tuple(out["dims"])
    if out["p"].shape != shape:
        raise ValueError("p has shape %s, settings say %s" % (out["p"].shape, shape))
    if out["costs"].shape != (out["iterations"] + 1, out["batch"]):
        raise ValueError("cost history does not match the iteration count")
    if (out["optimizer"] == "lbfgs") != (out["lbfgs_state"] is not None):
        raise ValueError("L-BFGS state missing or present for the wrong optimizer")
    return out
