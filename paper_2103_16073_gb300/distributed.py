"""Several GPUs on one sweep: independent (frequency, source) keys sharded
over ranks with no data-path collective.

Every frequency and source position of a sweep is a solve of its own
(Sec. 4 distributes a sweep over nodes frequency by frequency), so ranks
share nothing while they solve.  The keys are partitioned once, largest
predicted cost first (``fb_batch_partition`` in the library), each rank
solves its own keys and writes one result file per key, and after one
barrier rank 0 gathers the files.

Predicted cost of a key: N x predicted iterations.  FGMRES iteration counts
grow with the electrical size of the room; measured counts (17, 47 and 51
block-Jacobi iterations at kD ~ 81, 260 and 870) follow kD^(1/2) closely
enough to order the jobs, so the prediction is N x (kD)^(1/2).
"""
from __future__ import annotations

import math
import os

import numpy as np


def predicted_cost(n, k, diameter, nsrc=1):
    """N x (k D)^(1/2) per source: the predicted solve time of a key up to a
    constant (D: the room's diameter)."""
    return float(nsrc) * float(n) * math.sqrt(max(float(k) * float(diameter), 1.0))


def partition(costs, nranks):
    """Owner rank of every key and the load per rank (largest cost first to
    the least loaded rank; the library's host-only fb_batch_partition)."""
    import paper_2103_16073_gb300 as fb
    owner, load = fb.fb_batch_partition(costs, nranks)
    return owner.tolist(), load.tolist()


def rank_keys(owner, rank):
    """Indices of the keys a rank solves."""
    return [i for i, o in enumerate(owner) if o == rank]


def key_path(out_dir, key):
    return os.path.join(out_dir, "key_" + "_".join(str(int(v)) for v in key) + ".npz")


def write_result(out_dir, key, **arrays):
    """One result file per key, written under a temporary name and renamed
    so that a reader never sees a partial file."""
    os.makedirs(out_dir, exist_ok=True)
    path = key_path(out_dir, key)
    tmp = path + f".tmp{os.getpid()}.npz"
    np.savez(tmp, **arrays)
    os.replace(tmp, path)
    return path


def gather(out_dir, keys):
    """{key: {name: array}} of every key's result file (after the barrier
    that ends the solves of all ranks); raises if a key is missing."""
    out = {}
    for key in keys:
        path = key_path(out_dir, key)
        if not os.path.exists(path):
            raise FileNotFoundError(f"no result for key {key}: {path}")
        with np.load(path) as z:
            out[tuple(key)] = {name: z[name] for name in z.files}
    return out
