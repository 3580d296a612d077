"""Checkpoint / resume of a solve: the problem description, the factors and the sweep
history are written to one .npz file; resuming rebuilds the problem from the
description, loads the factors and continues the subspace iteration from them (the
paper keeps its solution as factors, and a slab boundary is a natural checkpoint).
Also a per-sweep JSON-lines log of a solve report."""
from __future__ import annotations

import json

import numpy as np


def save(path, desc, U, history=(), sweeps_done=0):
    """Write desc (JSON-serialisable apart from numpy arrays in nodal sources), the
    factors of U (a taps.Factors) and the history to path (.npz)."""
    facs = U.get()
    arrays = {f"U{d}": u for d, u in enumerate(facs)}
    # nodal source vectors travel as arrays; the rest of the description as JSON
    src = []
    for r, (beta, fl) in enumerate(desc["sources"]):
        row = []
        for d, (kind, par) in enumerate(fl):
            if kind == "nodal":
                key = f"src_{r}_{d}"
                arrays[key] = np.asarray(par, dtype=float)
                row.append([kind, key])
            elif kind == "opvec":
                key = f"src_{r}_{d}"
                arrays[key] = np.asarray(par[1], dtype=float)
                row.append([kind, [par[0], key]])
            else:
                row.append([kind, [float(v) for v in par]])
        src.append([float(beta), row])
    meta = dict(name=desc.get("name", ""), dims=desc["dims"], terms=[[float(a), list(o)] for a, o in desc["terms"]],
                sources=src, M=int(facs[0].shape[1]), D=len(facs), sweeps_done=int(sweeps_done),
                history=[list(map(float, h)) for h in history])
    np.savez(path, meta=np.frombuffer(json.dumps(meta).encode(), dtype=np.uint8), **arrays)


def load(path):
    """(description, factors list, sweeps_done, history) from a checkpoint."""
    z = np.load(path)
    meta = json.loads(bytes(z["meta"]).decode())
    sources = []
    for beta, row in meta["sources"]:
        fl = []
        for kind, par in row:
            if kind == "nodal":
                fl.append((kind, z[par]))
            elif kind == "opvec":
                fl.append((kind, (par[0], z[par[1]])))
            else:
                fl.append((kind, tuple(par)))
        sources.append((beta, fl))
    dims = [dict(dm, weight_poly=tuple(dm["weight_poly"])) for dm in meta["dims"]]
    desc = dict(name=meta["name"], dims=dims, terms=[(a, o) for a, o in meta["terms"]], sources=sources)
    facs = [z[f"U{d}"] for d in range(meta["D"])]
    return desc, facs, meta["sweeps_done"], [tuple(h) for h in meta["history"]]


def resume(path, stream=None):
    """A taps.Problem and taps.Factors restored from a checkpoint, ready to continue."""
    from . import taps
    desc, facs, done, hist = load(path)
    P = taps.Problem(desc, stream=stream)
    U = P.factors(facs[0].shape[1])
    U.set(facs)
    return P, U, done, hist


def write_history_jsonl(path, report):
    """One JSON line per sweep of a taps_solve report: mode count, factor change and
    residual."""
    with open(path, "w") as f:
        for i, (M, change, rho) in enumerate(report.get("history", [])):
            f.write(json.dumps(dict(sweep=i + 1, M=int(M), change=float(change), rho=float(rho))) + "\n")
