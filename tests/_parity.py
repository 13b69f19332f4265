"""Parity assertions of the GPU tests against the FP64 oracle.

Every vector output is held to two bounds on the same inputs:
  * norm-wise:     ||a - b|| / ||b|| < tol
  * element-wise:  max_i |a_i - b_i| <= elem * max_i |b_i|   (elem = tol unless given)
The norm bound alone lets a fault confined to a few entries pass (one entry
of a 128^3 grid wrong by 1 % moves the norm by ~7e-6); the element-wise bound
catches a wrong tile edge, a wrong packed kz = 0 / N/2 column or a wrong
pencil tile.  Scalars are held to |a - b| <= tol |b|.

With HM_PARITY_REPORT=<path> in the environment, every checked quantity with
its measured errors is written to that JSON file when the process exits
(the error table of the design notes is taken from it).
"""
import atexit
import json
import os

import numpy as np

_REPORT = []


def _flat(x):
    if hasattr(x, "detach"):
        x = x.detach().cpu().numpy()
    x = np.asarray(x).ravel()
    if np.iscomplexobj(x):
        x = np.concatenate([np.real(x), np.imag(x)])
    return x.astype(np.float64)


def rel(a, b):
    a, b = _flat(a), _flat(b)
    den = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (den if den > 0 else 1.0))


def maxrel(a, b):
    a, b = _flat(a), _flat(b)
    if a.size == 0:
        return 0.0
    den = np.max(np.abs(b))
    return float(np.max(np.abs(a - b)) / (den if den > 0 else 1.0))


def check(label, a, b, tol, elem=None):
    """Norm-wise and element-wise parity of a vector output."""
    r, m = rel(a, b), maxrel(a, b)
    e = tol if elem is None else elem
    _REPORT.append({"label": label, "norm_rel": r, "max_rel": m, "tol": tol, "elem_tol": e})
    assert r < tol, f"{label}: norm-wise relative error {r:.3e} >= {tol:.1e}"
    assert m <= e, f"{label}: element-wise error {m:.3e} x max|ref| > {e:.1e}"


def check_scalar(label, a, b, tol):
    a, b = float(a), float(b)
    err = abs(a - b) / (abs(b) if b != 0 else 1.0)
    _REPORT.append({"label": label, "rel": err, "tol": tol})
    assert err <= tol, f"{label}: relative error {err:.3e} > {tol:.1e} ({a!r} vs {b!r})"


def _write():
    path = os.environ.get("HM_PARITY_REPORT")
    if path and _REPORT:
        d = os.path.dirname(path)
        if d:
            os.makedirs(d, exist_ok=True)
        with open(path, "w") as fh:
            json.dump(_REPORT, fh, indent=1)


atexit.register(_write)
