"""Error paths of the C ABI on a GPU: validation before launch, bounded device failures."""
import numpy as np
import pytest

from paper_1708_06142_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _ts():
    from paper_1708_06142_gb300.treesolver import TreeSolver
    return TreeSolver(0)


def test_walk_before_build_and_bad_params():
    import torch
    from paper_1708_06142_gb300.treesolver import TSError
    ts = _ts()
    pot = torch.empty(512, device="cuda")
    acc = torch.empty(512, 3, device="cuda")
    ts.ncell = 512
    with pytest.raises(TSError) as e:
        ts.gravity_walk(pot, acc)
    assert e.value.status == 5
    mesh, rho = I.sphere_32(ncell_axis=8)
    ts.tree_build(mesh, torch.from_numpy(rho.reshape(-1)).cuda())
    for kw in (dict(theta=0.0), dict(theta=-1.0), dict(mac="ape", a_lim=0.0)):
        with pytest.raises(TSError) as e:
            ts.gravity_walk(pot, acc, **kw)
        assert e.value.status == 1


def test_malformed_meshes_rejected():
    import torch
    from paper_1708_06142_gb300.treesolver import TSError
    mesh, rho = I.sphere_32(ncell_axis=16)
    d = torch.from_numpy(rho.reshape(-1)).cuda()
    bad = []
    m = I.Mesh(mesh.level.copy(), mesh.child.copy(), mesh.lo.copy(), mesh.size.copy())
    m.child[0, 3] = -1                        # partial children
    bad.append(m)
    m = I.Mesh(mesh.level.copy(), mesh.child.copy(), mesh.lo.copy(), mesh.size.copy())
    m.lo[1, 0] += 0.01                        # child outside its octant
    bad.append(m)
    m = I.Mesh(mesh.level.copy(), mesh.child.copy(), mesh.lo.copy(), mesh.size.copy())
    m.level[2] = 5                            # wrong level
    bad.append(m)
    m = I.Mesh(mesh.level.copy(), mesh.child.copy(), mesh.lo.copy(), mesh.size.copy(), bc=(0, 1, 0))
    bad.append(m)
    ts = _ts()
    for k, m in enumerate(bad):
        with pytest.raises(TSError) as e:
            if k < 3:
                ts.tree_build(m, d)
            else:
                ts.tree_build(m, d)
                ts.ewald_field(16)
        assert e.value.status in (1, 2), k


def test_periodic_walk_needs_ewald_field():
    import torch
    from paper_1708_06142_gb300.treesolver import TSError
    mesh = I.uniform_mesh(8, bc=(1, 1, 1))
    ts = _ts()
    ts.tree_build(mesh, torch.ones(512, dtype=torch.float64, device="cuda"))
    with pytest.raises(TSError) as e:
        ts.gravity_walk(torch.empty(512, device="cuda"), torch.empty(512, 3, device="cuda"))
    assert e.value.status == 5


def test_stack_overflow_is_reported_not_hung():
    """A tree refined to level 19 towards the far corner: the refined branch is the last child at
    every level, so the depth-first stack keeps its 7 opened siblings per level (about 7 x 21 > 128
    entries for targets in the deepest block).  The kernel stops that warp's walk, latches
    TS_ERR_STACK_OVERFLOW, and the context stays usable."""
    import torch
    from paper_1708_06142_gb300.treesolver import TSError
    p = np.array([1.0, 1.0, 1.0]) - 1e-7

    def refine(lev, lo, sz):
        return lev < 19 and np.all(p >= lo) and np.all(p < lo + sz)

    mesh = I.build_mesh(refine)
    rho = np.ones((mesh.nleaf, 8, 8, 8))
    ts = _ts()
    ts.tree_build(mesh, torch.from_numpy(rho.reshape(-1)).cuda())
    pot = torch.empty(mesh.ncell, device="cuda")
    acc = torch.empty(mesh.ncell, 3, device="cuda")
    ts.gravity_walk(pot, acc, theta=0.01)
    with pytest.raises(TSError) as e:
        ts.sync()
    assert e.value.status == 6
    # the context still works on a shallow mesh afterwards
    mesh2, rho2 = I.sphere_32(ncell_axis=16)
    ts.tree_build(mesh2, torch.from_numpy(rho2.reshape(-1)).cuda())
    pot2 = torch.empty(mesh2.ncell, device="cuda")
    acc2 = torch.empty(mesh2.ncell, 3, device="cuda")
    ts.gravity_walk(pot2, acc2)
    ts.sync()
