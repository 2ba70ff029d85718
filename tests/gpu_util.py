"""Helpers shared by the GPU parity tests (inputs and metrics only; no method arithmetic)."""
import numpy as np


def e_a(a, aref, amax=None):
    """Relative acceleration error of eq. (ea): |a - a_ref| / a_ref,max."""
    if amax is None:
        amax = np.linalg.norm(aref, axis=1).max()
    return np.linalg.norm(a - aref, axis=1) / amax


def run_gravity(mesh, rho, precision="fp32", ewald_n=None, tpl=None, **kw):
    import torch
    from paper_1708_06142_gb300.treesolver import TreeSolver
    dev = torch.device("cuda:0")
    ts = TreeSolver(0)
    if tpl is not None:
        ts.set_walk_grouping(precision, tpl)
    ts.tree_build(mesh, torch.from_numpy(np.ascontiguousarray(rho).reshape(-1)).to(dev))
    if any(mesh.bc):
        ts.ewald_field(ewald_n or 64)
    dt = torch.float64 if precision == "fp64" else torch.float32
    pot = torch.empty(mesh.ncell, dtype=dt, device=dev)
    acc = torch.empty(mesh.ncell, 3, dtype=dt, device=dev)
    ts.gravity_walk(pot, acc, precision=precision, **kw)
    ts.sync()
    st = ts.stats()
    return ts, pot.cpu().numpy().astype(np.float64), acc.cpu().numpy().astype(np.float64), st
