"""Columns of a seeded schema as torch buffers for the engine's C ABI: device
tensors, or pinned host tensors for the host-input modes.  Marshalling only."""
from __future__ import annotations

import numpy as np


def to_device(schema, device='cuda:0') -> dict:
    """{(relation, column): device tensor} holding every column of `schema`."""
    import torch
    out = {}
    for r in schema.relations:
        for c in r.columns:
            out[(r.name, c.name)] = torch.from_numpy(np.ascontiguousarray(c.data)).to(device)
    return out


def to_pinned(schema) -> dict:
    """{(relation, column): pinned host tensor} holding every column of `schema`."""
    import torch
    out = {}
    for r in schema.relations:
        for c in r.columns:
            out[(r.name, c.name)] = torch.from_numpy(np.ascontiguousarray(c.data)).pin_memory()
    return out
