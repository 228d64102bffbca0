"""Persistent table of autotuned launch shapes, keyed by graph shape.

deco_autotune times the launch shapes of a phase on one graph and keeps the
winner with that graph handle.  This module stores those decisions in a JSON
file so that a later process (or a new handle of a graph with the same shape)
can install them with deco_set_tuning instead of timing again.

Key: GPU name, n, nnz, weighted flag, column count C, precision.
"""
from __future__ import annotations

import json
import os
from typing import Dict, Optional

from . import _lib as L


def _gpu_name() -> str:
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.get_device_name()
    except Exception:
        pass
    return "unknown"


def shape_key(g: L.Graph, C: int, precision: int) -> str:
    n, nnz, weighted = L.deco_graph_info(g)
    return f"{_gpu_name()}|n={n}|nnz={nnz}|w={weighted}|C={C}|p={precision}"


class TuningTable:
    def __init__(self, path: Optional[str] = None):
        self.path = path
        self.table: Dict[str, dict] = {}
        if path and os.path.exists(path):
            with open(path) as f:
                self.table = json.load(f)

    def save(self):
        if self.path:
            tmp = self.path + ".tmp"
            with open(tmp, "w") as f:
                json.dump(self.table, f, indent=1, sort_keys=True)
            os.replace(tmp, self.path)

    def ensure(self, g: L.Graph, C: int, precision: int, objective: int = L.DECO_OBJ_MULTILINEAR01,
               momentum: float = 0.9, probe_steps: int = 50) -> int:
        """Install the recorded shape for (g, C, precision), timing it first if unknown."""
        key = shape_key(g, C, precision)
        ent = self.table.get(key)
        if ent is not None:
            L.deco_set_tuning(g, C, precision, ent["kernel"])
            return ent["kernel"]
        sel, us = L.deco_autotune(g, C, precision, objective, momentum, probe_steps)
        self.table[key] = {"kernel": sel, "us_per_step": us}
        return sel
