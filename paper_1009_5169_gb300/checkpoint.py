"""Checkpoints: the gauge field, the pseudo-fermion sources and the trained
network's parameters in one file, with a header saying what each array is.

The file is a numpy .npz archive.  Its "header" entry is a JSON document:
the format tag and version, for each stored array its shape and dtype, and
the caller's metadata (seeds, lattice sizes, kappa, training state ...).
Arrays: "links" ([(T+1) L^3, 4, 3, 3] complex128, the canonical layout of
sf_lattice_create), "sources" ([nrhs, V/2, 4, 3] complex128), "cnn_params"
(the flat FP32 parameter array of sf_cnn_create, with "cnn_hidden").
Only the network's parameters are kept: a network loaded from a checkpoint
resumes training with fresh optimiser moments.
"""
from __future__ import annotations

import json
from typing import Optional

import numpy as np

FORMAT = "sf-gb300-checkpoint"
VERSION = 1


def save(path: str, *, links: Optional[np.ndarray] = None, sources: Optional[np.ndarray] = None,
         cnn_hidden: Optional[int] = None, cnn_params: Optional[np.ndarray] = None,
         meta: Optional[dict] = None) -> None:
    """Write the given arrays and metadata to path (an .npz archive)."""
    arrays = {}
    if links is not None:
        arrays["links"] = np.ascontiguousarray(links, dtype=np.complex128)
    if sources is not None:
        arrays["sources"] = np.ascontiguousarray(sources, dtype=np.complex128)
    if (cnn_params is None) != (cnn_hidden is None):
        raise ValueError("cnn_params and cnn_hidden go together")
    if cnn_params is not None:
        arrays["cnn_params"] = np.ascontiguousarray(cnn_params, dtype=np.float32).reshape(-1)
    header = {"format": FORMAT, "version": VERSION,
              "arrays": {k: {"shape": list(v.shape), "dtype": str(v.dtype)} for k, v in arrays.items()},
              "cnn_hidden": cnn_hidden, "meta": meta or {}}
    with open(path, "wb") as f:
        np.savez(f, header=np.frombuffer(json.dumps(header).encode(), dtype=np.uint8), **arrays)


def load(path: str) -> dict:
    """Read a checkpoint: a dict with "meta", "cnn_hidden" and whichever of
    "links", "sources", "cnn_params" it holds.  Raises ValueError on a file
    that is not such a checkpoint or whose arrays do not match its header."""
    with np.load(path, allow_pickle=False) as z:
        if "header" not in z.files:
            raise ValueError(f"{path}: no checkpoint header")
        header = json.loads(bytes(z["header"]).decode())
        if header.get("format") != FORMAT:
            raise ValueError(f"{path}: not a {FORMAT} file")
        if header.get("version") != VERSION:
            raise ValueError(f"{path}: version {header.get('version')}, this library reads {VERSION}")
        out = {"meta": header.get("meta", {}), "cnn_hidden": header.get("cnn_hidden")}
        for name, desc in header["arrays"].items():
            a = z[name]
            if list(a.shape) != desc["shape"] or str(a.dtype) != desc["dtype"]:
                raise ValueError(f"{path}: array {name} does not match its header")
            out[name] = a
    return out


def save_cnn(path: str, cnn, meta: Optional[dict] = None, **arrays) -> None:
    """save() with a binding.Cnn's hidden width and current parameters."""
    save(path, cnn_hidden=cnn.hidden, cnn_params=cnn.params(), meta=meta, **arrays)


def load_cnn(path: str, device: int = 0):
    """A binding.Cnn built from the parameters of a checkpoint."""
    from . import binding
    c = load(path)
    if "cnn_params" not in c:
        raise ValueError(f"{path}: holds no network parameters")
    return binding.Cnn(int(c["cnn_hidden"]), c["cnn_params"], device=device)
