"""Launch-shape cache for the autotuner.

A JSON file maps a lattice's shape class and the library build to the best
launch shape the autotuner found for it, so that a program tuning the same
shape again takes the stored shape instead of timing every candidate.  The
key holds what the timings depend on: storage form, D and extents,
boundary and glued directions, sublattice cut, whether two couplings are in
use, the number of chains of a fused launch, and the library's version
string (which names the GPU architecture it was built for).  Plain host
code: it reads and writes the file and nothing else.
"""
from __future__ import annotations

import json
import os
import tempfile


def key_of(configs, version: str) -> str:
    """Cache key of one lattice (a list of one config) or a fused ensemble."""
    parts = [version, f"n{len(configs)}"]
    for c in configs[:1] if len({_shape(c) for c in configs}) == 1 else configs:
        parts.append(_shape(c))
    return "|".join(parts)


def _shape(c) -> str:
    dims = "x".join(str(c.dims[k]) for k in range(c.D))
    ndiv = "x".join(str(max(1, c.ndiv[k])) for k in range(c.D))
    two = int(c.beta1 >= 0.0 and c.beta1 != c.beta)
    return f"s{c.storage}:D{c.D}:{dims}:b{c.boundary}:g{c.glue_mask}:div{ndiv}:w{two}"


def lookup(path: str, key: str):
    """The stored (variant, threads, ctas_per_sm, us_per_sweep), or None."""
    try:
        with open(path) as f:
            entry = json.load(f).get(key)
    except (OSError, ValueError):
        return None
    if not entry:
        return None
    return int(entry["variant"]), int(entry["threads"]), int(entry["ctas_per_sm"]), float(entry["us_per_sweep"])


def store(path: str, key: str, shape) -> None:
    """Add or replace one entry; the file is replaced atomically."""
    try:
        with open(path) as f:
            table = json.load(f)
    except (OSError, ValueError):
        table = {}
    v, t, c, us = shape
    table[key] = {"variant": int(v), "threads": int(t), "ctas_per_sm": int(c), "us_per_sweep": float(us)}
    d = os.path.dirname(os.path.abspath(path))
    fd, tmp = tempfile.mkstemp(dir=d, prefix=".su3tune")
    with os.fdopen(fd, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)
    os.replace(tmp, path)
