"""Force-error measures shared by the GPU parity tests (no GPU needed here).

Two measures of the per-particle force error against the FP64 oracle:

* the tested one, |F_i - F_i^oracle| / S_i with S_i = sum_j |F_ij| the sum of
  the pair-force magnitudes of particle i: the scale against which any
  floating-point evaluation of F_i = sum_j F_ij is conditioned (where the pair
  forces cancel, |F_i| << S_i and no finite precision meets a flat relative
  bound on |F_i|);
* the plain relative error, reported beside it: |dF_i| / max(|F_i|, 1e-3 F_rms)
  (a floor at 1e-3 of the RMS force), its unfloored maximum over the particles
  with |F_i| >= F_rms, and max |dF_i| / F_rms.

`report` prints the figures and, when the environment variable
LJMD_PARITY_REPORT names a file, appends them to it as one JSON line.
"""
import json
import os

import numpy as np

import oracle


def pair_scale(box, pos, lj, types=None):
    """S_i = sum_j |F_ij| over pairs within the cutoff (oracle pair function)."""
    from scipy.spatial import cKDTree
    n = pos.shape[0]
    t = np.zeros(n, np.int32) if types is None else types
    tree = cKDTree(np.mod(pos, box), boxsize=box)
    pairs = tree.query_pairs(float(lj.rcut.max()) + 1e-9, output_type="ndarray")
    d = pos[pairs[:, 0]] - pos[pairs[:, 1]]
    d -= box * np.rint(d / box)
    r2 = np.sum(d * d, axis=1)
    S = np.zeros(n)
    for k, (i, j) in enumerate(pairs):
        f = oracle.pair(lj.eps[t[i], t[j]], lj.sigma[t[i], t[j]], lj.rcut[t[i], t[j]], 1, r2[k])[0]
        m = abs(f) * np.sqrt(r2[k])
        S[i] += m
        S[j] += m
    return S


def figures(f, fo, S=None):
    """Force-error figures of f against the oracle's fo (n x 3 each)."""
    f = np.asarray(f, dtype=np.float64).reshape(-1, 3)
    fo = np.asarray(fo, dtype=np.float64).reshape(-1, 3)
    df = np.linalg.norm(f - fo, axis=1)
    mag = np.linalg.norm(fo, axis=1)
    frms = float(np.sqrt(np.mean(mag ** 2))) if mag.size else 0.0
    out = {"n": int(mag.size), "F_rms": frms}
    if mag.size and frms > 0:
        out["rel_floored_max"] = float((df / np.maximum(mag, 1e-3 * frms)).max())
        big = mag >= frms
        out["rel_unfloored_max_over_F_ge_Frms"] = float((df[big] / mag[big]).max()) if big.any() else None
        out["abs_max_over_Frms"] = float(df.max() / frms)
    if S is not None and mag.size:
        out["max_over_S"] = float((df / np.asarray(S)).max())
    return out


def report(name, fig):
    line = dict(fig, case=name)
    print("force-error", json.dumps(line))
    path = os.environ.get("LJMD_PARITY_REPORT")
    if path:
        with open(path, "a") as fh:
            fh.write(json.dumps(line) + "\n")
