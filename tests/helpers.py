"""Shared test helpers: build the oracle and the GPU handle from the same ProblemSpec."""
import numpy as np


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def gpu_handle(spec):
    from paper_2603_25233_gb300.api import Handle
    return Handle(spec)


def oracle_disc(spec):
    from oracle.dg import Discretisation
    return Discretisation.from_spec(spec)
