"""ctypes front end of the FP64 CPU oracle (oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, by __graft_entry__.smoke() and by bench.py's
CPU-baseline and reference legs.  The CUDA library never imports, links or calls this module.
The shared object is compiled from oracle.c with gcc on first use (or by build()).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "_oracle.so")
_lock = threading.Lock()
_lib = None

NB = 8
NCB = 512


def build(force: bool = False) -> str:
    """Compile oracle.c into _oracle.so (gcc, OpenMP, no -ffast-math)."""
    with _lock:
        stale = (not os.path.exists(_LIB)) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC)
        if force or stale:
            tmp = _LIB + f".{os.getpid()}.tmp"
            subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fopenmp", "-fPIC", "-shared",
                                   "-fno-fast-math", "-ffp-contract=off", _SRC, "-o", tmp, "-lm"])
            os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        P = C.c_void_p
        i32, i64, f64 = C.c_int, C.c_int64, C.c_double
        L.or_tree_build.argtypes = [i32, P, P, P, P, P, P, P, P, P, P, P]
        L.or_tree_bmoments.argtypes = [i32, P, P, P, P, P, P, P, P]
        L.or_gravity_walk.argtypes = [i32, P, P, P, P, P, P, i32, f64, f64, f64, f64, i32, P, i32, P,
                                      i64, P, P, P, P]
        L.or_direct_sum.argtypes = [i32, P, P, P, P, P, P, f64, i64, P, P, P]
        L.or_gravity_walk_sumsq.argtypes = [i32, P, P, P, P, P, P, f64, f64, f64, i32, i64, P, P, P, P]
        L.or_itilde_2p1i.argtypes = [f64, f64, f64, P, P]
        L.or_km_1p2i.argtypes = [f64, f64, f64, P, P]
        L.or_ewald.argtypes = [P, P, f64, f64, f64, i32, i64, P, P, P]
        L.or_ewald_far.argtypes = [P, P, f64, i64, P, P, P]
        L.or_ewald_table.argtypes = [P, P, f64, i32, P, P]
        L.or_ewald_taylor_table.argtypes = [P, P, f64, i32, f64, P, P]
        L.or_healpix_vec2pix.argtypes = [i32, i64, P, P]
        L.or_healpix_pix2ang.argtypes = [i32, i64, P, P, P]
        L.or_noderay_table.argtypes = [i32, i32, i32, i32, f64, f64, i32, P]
        L.or_column_walk.argtypes = [i32, P, P, P, P, P, P, f64, f64, f64, i32, i32, i32, i32, f64, f64,
                                     i32, P, i64, P, P, P]
        L.or_column_walk_q.argtypes = [i32, P, P, P, P, P, i32, P, P, f64, f64, f64, i32, i32, i32, i32, f64,
                                       f64, i32, P, i64, P, P, P]
        L.or_num_threads.restype = C.c_int
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def _mesh_args(mesh, rho):
    level = np.ascontiguousarray(mesh.level, dtype=np.int32)
    child = np.ascontiguousarray(mesh.child, dtype=np.int32)
    lo = np.ascontiguousarray(mesh.lo, dtype=np.float64)
    size = np.ascontiguousarray(mesh.size, dtype=np.float64)
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    assert rho.size == mesh.nleaf * NCB
    keep = (level, child, lo, size, rho)
    return keep, [mesh.nblocks, _p(level), _p(child), _p(lo), _p(size), _p(rho)]


def num_threads() -> int:
    return int(lib().or_num_threads())


def tree_build(mesh, rho):
    """Per-block (M, CoM) and per-leaf block-tree nodes (level 1: [nleaf,8], level 2: [nleaf,64])."""
    keep, args = _mesh_args(mesh, rho)
    nb, nl = mesh.nblocks, mesh.nleaf
    bm, bc = np.zeros(nb), np.zeros((nb, 3))
    n1m, n1c = np.zeros((nl, 8)), np.zeros((nl, 8, 3))
    n2m, n2c = np.zeros((nl, 64)), np.zeros((nl, 64, 3))
    rc = lib().or_tree_build(*args, _p(bm), _p(bc), _p(n1m), _p(n1c), _p(n2m), _p(n2c))
    assert rc == 0
    return dict(block_mass=bm, block_com=bc, n1_mass=n1m, n1_com=n1c, n2_mass=n2m, n2_com=n2c)


def tree_bmoments(mesh, rho):
    """MPE moments B_p = sum_i m_i |r_i - r_a|^p (p = 2, 3) per node by direct sums over the node's
    cells: blocks [nb, 2], level-1 nodes [nleaf, 8, 2], level-2 nodes [nleaf, 64, 2]."""
    keep, args = _mesh_args(mesh, rho)
    bb = np.zeros((mesh.nblocks, 2))
    n1, n2 = np.zeros((mesh.nleaf, 8, 2)), np.zeros((mesh.nleaf, 64, 2))
    rc = lib().or_tree_bmoments(*args, _p(bb), _p(n1), _p(n2))
    assert rc == 0
    return dict(block=bb, n1=n1, n2=n2)


def gravity_walk(mesh, rho, targets=None, mac="bh", theta=0.5, safe_box=1.2, a_lim=0.0, G=1.0,
                 ewald="series", table=None, queue_max=4096):
    """FP64 tree walk.  Returns (pot[nt], acc[nt,3], counts{interactions, mac_tests}).
    mac="sumsq": the SumSquare MAC (priority-queue walk, exact Ewald series on periodic axes);
    a_lim limits the root of the frontier's summed squared MPE bounds; counts adds the number of
    targets whose queue of at most queue_max nodes filled ("overflows")."""
    keep, args = _mesh_args(mesh, rho)
    if targets is None:
        targets = np.arange(mesh.ncell, dtype=np.int64)
    targets = np.ascontiguousarray(targets, dtype=np.int64)
    bc = np.asarray(mesh.bc, dtype=np.int32)
    nt = targets.size
    pot, acc, cnt = np.zeros(nt), np.zeros((nt, 3)), np.zeros(3, dtype=np.int64)
    if mac == "sumsq":
        rc = lib().or_gravity_walk_sumsq(*args, _p(bc), safe_box, a_lim, G, queue_max, nt, _p(targets), _p(pot),
                                         _p(acc), _p(cnt))
        assert rc == 0, rc
        return pot, acc, dict(interactions=int(cnt[0]), mac_tests=int(cnt[1]), overflows=int(cnt[2]))
    tab = text = None
    tn = 0
    if ewald in ("table", "taylor"):
        tab, text = table
        tab = np.ascontiguousarray(tab, dtype=np.float64)
        text = np.ascontiguousarray(text, dtype=np.float64)
        tn = tab.shape[0]
    rc = lib().or_gravity_walk(*args, _p(bc), {"bh": 0, "ape": 1, "mpe": 2}[mac], theta, safe_box, a_lim, G,
                               {"series": 0, "table": 1, "taylor": 2}[ewald], _p(tab), tn, _p(text), nt, _p(targets),
                               _p(pot), _p(acc), _p(cnt))
    assert rc == 0, rc
    return pot, acc, dict(interactions=int(cnt[0]), mac_tests=int(cnt[1]))


def direct_sum(mesh, rho, targets=None, G=1.0):
    """O(N^2) reference: every target against every other cell (Ewald series on periodic axes)."""
    keep, args = _mesh_args(mesh, rho)
    if targets is None:
        targets = np.arange(mesh.ncell, dtype=np.int64)
    targets = np.ascontiguousarray(targets, dtype=np.int64)
    bc = np.asarray(mesh.bc, dtype=np.int32)
    nt = targets.size
    pot, acc = np.zeros(nt), np.zeros((nt, 3))
    rc = lib().or_direct_sum(*args, _p(bc), G, nt, _p(targets), _p(pot), _p(acc))
    assert rc == 0, rc
    return pot, acc


def ewald(bc, L, d, corr=False, alpha_lx=2.0, rcut2=15.0, kcut2=10.0):
    """phi and A = -grad phi of one unit mass with its periodic images (or the smooth correction)."""
    bc = np.asarray(bc, dtype=np.int32)
    L = np.asarray(L, dtype=np.float64)
    d = np.ascontiguousarray(np.atleast_2d(d), dtype=np.float64)
    n = d.shape[0]
    phi, A = np.zeros(n), np.zeros((n, 3))
    rc = lib().or_ewald(_p(bc), _p(L), alpha_lx, rcut2, kcut2, int(corr), n, _p(d), _p(phi), _p(A))
    assert rc == 0, rc
    return phi, A


def fourier_2p1i(s, gam, zeta):
    """The oracle's 2P1I Fourier factor (It, Ip) = (exp(-zeta s^2) I(s, gam), d/dgam of it), with I
    of eq. intdef in the closed forms of eqs. intij / int00 (s = sqrt(l1^2 + (l2/b)^2), gam >= 0)."""
    a, b = np.zeros(1), np.zeros(1)
    lib().or_itilde_2p1i(float(s), float(gam), float(zeta), _p(a), _p(b))
    return float(a[0]), float(b[0])


def km_1p2i(l1, eta, zeta):
    """The oracle's 1P2I integrals (K, M) of eq. int00p1 and its radial derivative's integral, by
    composite Gauss-Legendre quadrature (K(0, .) regularised as (J0 - 1) e^{-zeta q^2}/q)."""
    a, b = np.zeros(1), np.zeros(1)
    lib().or_km_1p2i(float(l1), float(eta), float(zeta), _p(a), _p(b))
    return float(a[0]), float(b[0])


def ewald_far(bc, L, d, alpha_lx=2.0):
    bc = np.asarray(bc, dtype=np.int32)
    L = np.asarray(L, dtype=np.float64)
    d = np.ascontiguousarray(np.atleast_2d(d), dtype=np.float64)
    n = d.shape[0]
    phi, A = np.zeros(n), np.zeros((n, 3))
    rc = lib().or_ewald_far(_p(bc), _p(L), alpha_lx, n, _p(d), _p(phi), _p(A))
    assert rc == 0, rc
    return phi, A


def ewald_table(bc, L, n=64, alpha_lx=2.0):
    """(table[n,n,n,4] of (C, A_c), extent[3]) on the folded grid."""
    bc = np.asarray(bc, dtype=np.int32)
    L = np.asarray(L, dtype=np.float64)
    tab, ext = np.zeros((n, n, n, 4)), np.zeros(3)
    rc = lib().or_ewald_table(_p(bc), _p(L), alpha_lx, n, _p(tab), _p(ext))
    assert rc == 0, rc
    return tab, ext


def ewald_taylor_table(bc, L, n=64, alpha_lx=2.0, eps=1e-5):
    """(table[n,n,n,10] of (C, A_c, Jxx, Jxy, Jxz, Jyy, Jyz, Jzz), extent[3]): the first-order Taylor
    table of Sec. 2.2.5 (approach 2); J = dA_c/dd by central differences with step eps * Lx."""
    bc = np.asarray(bc, dtype=np.int32)
    L = np.asarray(L, dtype=np.float64)
    tab, ext = np.zeros((n, n, n, 10)), np.zeros(3)
    rc = lib().or_ewald_taylor_table(_p(bc), _p(L), alpha_lx, n, eps * L[0], _p(tab), _p(ext))
    assert rc == 0, rc
    return tab, ext


def healpix_vec2pix(nside, v):
    v = np.ascontiguousarray(np.atleast_2d(v), dtype=np.float64)
    pix = np.zeros(v.shape[0], dtype=np.int64)
    lib().or_healpix_vec2pix(nside, v.shape[0], _p(v), _p(pix))
    return pix


def healpix_pix2ang(nside, pix):
    pix = np.ascontiguousarray(pix, dtype=np.int64)
    z, phi = np.zeros(pix.size), np.zeros(pix.size)
    lib().or_healpix_pix2ang(nside, pix.size, _p(pix), _p(z), _p(phi))
    return z, phi


NODERAY_DEFAULT = dict(ntheta=25, nphi=50, npsi=25, psi_min=1e-3, psi_max=1.0, nsub=8)


def noderay_table(nside, ntheta=25, nphi=50, npsi=25, psi_min=1e-3, psi_max=1.0, nsub=8):
    npix = 12 * nside * nside
    w = np.zeros((ntheta, nphi, npsi, npix))
    lib().or_noderay_table(nside, ntheta, nphi, npsi, psi_min, psi_max, nsub, _p(w))
    return w


def column_av(cols, k=1.0):
    """Mean visual extinction per cell (Sec. 2.3, eq. av): A_V = -(1/2.5) ln[(1/N_PIX) sum_i
    exp(-2.5 k N_i)] over the cell's HEALPix column map cols[..., N_PIX]; k converts the map's
    column unit into units of 1.87e21 cm^-2.  FP64, the definition as written."""
    x = np.asarray(cols, dtype=np.float64)
    return -np.log(np.mean(np.exp(-2.5 * k * x), axis=-1)) / 2.5


def h2_self_shielding(n_h2, b5=3.0):
    """H2 self-shielding factor of one column N_H2 [cm^-2] (Draine & Bertoldi 1996, their eq. 37, the
    form the paper's chemistry takes from Glover & Mac Low 2007):
        f = 0.965 / (1 + x / b5)^2 + 0.035 / sqrt(1 + x) exp(-8.5e-4 sqrt(1 + x)),  x = N_H2 / 5e14,
    b5 the Doppler parameter in km/s."""
    x = np.asarray(n_h2, dtype=np.float64) / 5e14
    return 0.965 / (1.0 + x / b5) ** 2 + 0.035 / np.sqrt(1.0 + x) * np.exp(-8.5e-4 * np.sqrt(1.0 + x))


def column_shielding(cols, k_av=1.0, k_h2=1.0, b5=3.0, k_co=1.0, co_table=None, lg_co=(0.0, 1.0), lg_h2=(0.0, 1.0)):
    """Pixel averages of the shielding quantities of one cell from its l_q = 3 maps
    cols[..., 3, N_PIX] (total, H2, CO columns), built like eq. av (Sec. 2.3: the coefficients are
    'computed by averaging over the Healpix maps in a similar way'):
      A_V      = -(1/2.5) ln[ mean_i exp(-2.5 k_av N_i) ]                           (eq. av)
      <f_H2>   = mean_i f_DB96(k_h2 N_H2,i)                                         (h2_self_shielding)
      <f_CO>   = mean_i T(log10 k_co N_CO,i, log10 k_h2 N_H2,i), T bilinear in a table over
                 [lg_co] x [lg_h2] (co_table [n_co, n_h2], clamped at its edges; 1 without a table).
    FP64, the definitions as written.  Returns [..., 3]."""
    x = np.asarray(cols, dtype=np.float64)
    av = column_av(x[..., 0, :], k_av)
    nh2 = k_h2 * x[..., 1, :]
    fh2 = h2_self_shielding(nh2, b5).mean(-1)
    if co_table is None:
        fco = np.ones_like(fh2)
    else:
        T = np.asarray(co_table, dtype=np.float64)
        nco_, nh2_ = T.shape

        def coord(lg, lo, hi, n):
            u = (lg - lo) / (hi - lo) * (n - 1)
            u = np.clip(u, 0.0, n - 1.0)
            i = np.minimum(np.floor(u).astype(int), n - 2)
            return i, u - i

        with np.errstate(divide="ignore"):
            ic, fc = coord(np.log10(np.maximum(k_co * x[..., 2, :], 1e-300)), lg_co[0], lg_co[1], nco_)
            ih, fh = coord(np.log10(np.maximum(nh2, 1e-300)), lg_h2[0], lg_h2[1], nh2_)
        v = (T[ic, ih] * (1 - fc) * (1 - fh) + T[ic + 1, ih] * fc * (1 - fh) + T[ic, ih + 1] * (1 - fc) * fh +
             T[ic + 1, ih + 1] * fc * fh)
        fco = v.mean(-1)
    return np.stack([av, fh2, fco], -1)


def column_walk(mesh, rho, targets=None, nside=2, theta=0.5, safe_box=1.2, max_dist=1e99,
                table="default", ntheta=25, nphi=50, npsi=25, psi_min=1e-3, psi_max=1.0, nsub=8, quantities=None):
    """Per-target HEALPix column map [nt, 12 nside^2].  table=None: per-node sub-cube quadrature.
    quantities: None, or the densities [nq, ncell] (nq <= 2) of extra mapped quantities; the maps are
    then [nt, 1 + nq, 12 nside^2] (total mass first)."""
    if quantities is not None:
        return _column_walk_q(mesh, rho, quantities, targets, nside, theta, safe_box, max_dist, table, ntheta, nphi,
                              npsi, psi_min, psi_max, nsub)
    keep, args = _mesh_args(mesh, rho)
    if targets is None:
        targets = np.arange(mesh.ncell, dtype=np.int64)
    targets = np.ascontiguousarray(targets, dtype=np.int64)
    bc = np.asarray(mesh.bc, dtype=np.int32)
    if isinstance(table, str):
        table = noderay_table(nside, ntheta, nphi, npsi, psi_min, psi_max, nsub)
    if table is not None:
        table = np.ascontiguousarray(table, dtype=np.float64)
    npix = 12 * nside * nside
    cols = np.zeros((targets.size, npix))
    cnt = np.zeros(1, dtype=np.int64)
    rc = lib().or_column_walk(*args, _p(bc), theta, safe_box, max_dist, nside, ntheta, nphi, npsi,
                              psi_min, psi_max, nsub, _p(table), targets.size, _p(targets), _p(cols),
                              _p(cnt))
    assert rc == 0, rc
    return cols, dict(interactions=int(cnt[0]))


def _column_walk_q(mesh, rho, q, targets, nside, theta, safe_box, max_dist, table, ntheta, nphi, npsi, psi_min,
                   psi_max, nsub):
    keep, args = _mesh_args(mesh, rho)
    q = np.ascontiguousarray(np.asarray(q, dtype=np.float64).reshape(-1, mesh.ncell))
    nq = q.shape[0]
    assert nq <= 2
    if targets is None:
        targets = np.arange(mesh.ncell, dtype=np.int64)
    targets = np.ascontiguousarray(targets, dtype=np.int64)
    bc = np.asarray(mesh.bc, dtype=np.int32)
    if isinstance(table, str):
        table = noderay_table(nside, ntheta, nphi, npsi, psi_min, psi_max, nsub)
    if table is not None:
        table = np.ascontiguousarray(table, dtype=np.float64)
    npix = 12 * nside * nside
    cols = np.zeros((targets.size, 1 + nq, npix))
    cnt = np.zeros(1, dtype=np.int64)
    rc = lib().or_column_walk_q(*args, nq, _p(q), _p(bc), theta, safe_box, max_dist, nside, ntheta, nphi, npsi,
                                psi_min, psi_max, nsub, _p(table), targets.size, _p(targets), _p(cols), _p(cnt))
    assert rc == 0, rc
    return cols, dict(interactions=int(cnt[0]))


def error_stats(pot=None, acc=None, pot_ref=None, acc_ref=None, mod_const=False):
    """Accuracy of a solution against a reference (Sec. 3, eq. ea, and the same construction for the
    potential), in FP64 with numpy:
      e_a(c)   = |a(c) - a_ref(c)| / max_c' |a_ref(c')|
      e_phi(c) = |phi(c) - phi_ref(c)| / max_c' |phi_ref(c')|,
    where with mod_const each potential is first reduced by its own mean (periodic and mixed
    boundaries define the potential up to a constant).  A reference that is identically zero
    normalises by 1.  Returns the median and 99th percentile (numpy's linear interpolation at
    position q (n - 1)), the maximum, the normalisers and the count of non-finite errors."""
    out = {"n": 0, "n_nonfinite": 0, "a_ref_max": 0.0, "phi_ref_max": 0.0, "e_a_median": 0.0, "e_a_p99": 0.0,
           "e_a_max": 0.0, "e_phi_median": 0.0, "e_phi_p99": 0.0, "e_phi_max": 0.0}
    e_a = e_phi = None
    if acc is not None:
        acc = np.asarray(acc, dtype=np.float64).reshape(-1, 3)
        acc_ref = np.asarray(acc_ref, dtype=np.float64).reshape(-1, 3)
        amax = float(np.sqrt((acc_ref ** 2).sum(1)).max())
        e_a = np.sqrt(((acc - acc_ref) ** 2).sum(1)) / (amax if amax > 0 else 1.0)
        out.update(n=acc.shape[0], a_ref_max=amax, e_a_median=float(np.quantile(e_a, 0.5)),
                   e_a_p99=float(np.quantile(e_a, 0.99)), e_a_max=float(e_a.max()))
    if pot is not None:
        pot = np.asarray(pot, dtype=np.float64).reshape(-1)
        pot_ref = np.asarray(pot_ref, dtype=np.float64).reshape(-1)
        if mod_const:
            pot, pot_ref = pot - pot.mean(), pot_ref - pot_ref.mean()
        pmax = float(np.abs(pot_ref).max())
        e_phi = np.abs(pot - pot_ref) / (pmax if pmax > 0 else 1.0)
        out.update(n=pot.shape[0], phi_ref_max=pmax, e_phi_median=float(np.quantile(e_phi, 0.5)),
                   e_phi_p99=float(np.quantile(e_phi, 0.99)), e_phi_max=float(e_phi.max()))
    out["n_nonfinite"] = int(sum((~np.isfinite(e)).sum() for e in (e_a, e_phi) if e is not None))
    return out


def abu_corner_cells(nleaf):
    """Flat indices of the 8 corner cells (i, j, k in {0, 7}) of every leaf-block, [nleaf, 8]."""
    c = [k * 64 + j * 8 + i for k in (0, 7) for j in (0, 7) for i in (0, 7)]
    return (np.arange(nleaf, dtype=np.int64)[:, None] * NCB + np.asarray(c, dtype=np.int64)[None, :])


def abu_walk(mesh, rho, pot_old, acc_old, a_tol, phi_tol=0.0, **walk):
    """Adaptive Block Update (Sec. 2.2.6), in the paper's order: walk the 8 corner cells of every
    leaf-block; a block whose corner accelerations all differ from the previous values by less than
    a_tol (and, if phi_tol > 0, whose corner potentials differ by less than phi_tol) keeps its
    previous values in every cell; every other block is walked in full.  Returns (pot, acc,
    updated[nleaf] bool, interactions[nleaf] of the full walks)."""
    nl = mesh.nleaf
    corners = abu_corner_cells(nl)
    pc, ac, _ = gravity_walk(mesh, rho, corners.reshape(-1), **walk)
    pc, ac = pc.reshape(nl, 8), ac.reshape(nl, 8, 3)
    pot_old = np.asarray(pot_old, dtype=np.float64).reshape(-1)
    acc_old = np.asarray(acc_old, dtype=np.float64).reshape(-1, 3)
    da = np.linalg.norm(ac - acc_old[corners], axis=2)
    keep = np.all(da < a_tol, axis=1)
    if phi_tol > 0:
        keep &= np.all(np.abs(pc - pot_old[corners]) < phi_tol, axis=1)
    pot, acc = pot_old.copy(), acc_old.copy()
    nint = np.zeros(nl, dtype=np.int64)
    for n in np.nonzero(~keep)[0]:
        cells = np.arange(n * NCB, (n + 1) * NCB, dtype=np.int64)
        p, a, cnt = gravity_walk(mesh, rho, cells, **walk)
        pot[cells], acc[cells] = p, a
        nint[n] = cnt["interactions"]
    return pot, acc, ~keep, nint


def workload_update(w_prev, nint, tau=10.0, omega=8.0):
    """Block workload weight of Sec. 2.2.6: W = W_prev e^(-1/tau) + (1 - e^(-1/tau)) (2 + omega N / N_max),
    N the interactions of the block's last walk and N_max the largest over the leaf-blocks."""
    nint = np.asarray(nint, dtype=np.float64)
    nmax = nint.max() if nint.size and nint.max() > 0 else 1.0
    f = np.exp(-1.0 / tau)
    return np.asarray(w_prev, dtype=np.float64) * f + (1 - f) * (2 + omega * nint / nmax)


def _cell_keys(mesh):
    """Depth d of every cell (root block depth 0, cells 3 deeper than their block) and its integer
    position among the 2^d cells per axis of that depth, in the flat cell order [ncell]."""
    lf = mesh.leaves
    d_leaf = mesh.level[lf].astype(np.int64) + 2
    lo = (mesh.lo[lf] - mesh.domain_lo) / mesh.domain_size            # [nleaf, 3] in units of the domain
    base = np.rint(lo * np.ldexp(1.0, d_leaf)[:, None]).astype(np.int64)
    k, j, i = np.meshgrid(np.arange(NB), np.arange(NB), np.arange(NB), indexing="ij")
    loc = np.stack([i.reshape(-1), j.reshape(-1), k.reshape(-1)], 1)   # flat order: x fastest
    pos = (base[:, None, :] + loc[None, :, :]).reshape(-1, 3)
    dep = np.repeat(d_leaf, NCB)
    return dep, pos


def _key(dep, pos):
    return (np.asarray(dep, dtype=np.int64) << 57) | (pos[..., 0] << 38) | (pos[..., 1] << 19) | pos[..., 2]


def num_diff(mesh, pot):
    """Acceleration by numerical differentiation of a cell-centred potential (Sec. 2.2.2, the
    alternative to eq. accel), plain numpy in FP64.  For every cell and axis k:
        a_k = -(g(+1) - g(-1)) / (2 dx_k),
    g(m) the potential of the cube D(m) of the cell's own size m cells away along k: the value of the
    leaf cell containing D(m) if that cell is as large or larger, else the volume-weighted mean of
    the leaf cells inside D(m).  Periodic axes wrap D(m); where D(-1) or D(+1) lies outside the
    domain on an isolated axis, the one-sided a_k = -(-3 phi_0 + 4 g(+1) - g(+2)) / (2 dx_k)
    (mirrored at the upper edge) is used.  pot: [ncell] in the flat cell order; returns [ncell, 3]."""
    pot = np.asarray(pot, dtype=np.float64).reshape(-1)
    dep, pos = _cell_keys(mesh)
    assert dep.max() <= 18, "keys hold 19 bits per axis"
    dx = np.repeat(mesh.size[mesh.leaves] / NB, NCB, axis=0)              # [ncell, 3]
    leaf_keys = _key(dep, pos)
    order = np.argsort(leaf_keys)
    sorted_keys = leaf_keys[order]
    vol = np.ldexp(1.0, -3 * dep)                                         # cell volumes in domain units
    # volume-weighted sums over every ancestor cube that is not itself a leaf cell
    anc = {}
    for a in range(int(dep.min()), int(dep.max())):
        sel = dep > a
        if not sel.any():
            continue
        k = _key(np.full(sel.sum(), a), pos[sel] >> (dep[sel] - a)[:, None])
        u, inv = np.unique(k, return_inverse=True)
        anc[a] = (u, np.bincount(inv, weights=vol[sel] * pot[sel]), np.bincount(inv, weights=vol[sel]))

    def guard(m, axis):
        """(value, present) of the guard cubes at offset m along axis for every cell."""
        q = pos.copy()
        q[:, axis] += m
        n = np.int64(1) << dep
        out = (q[:, axis] < 0) | (q[:, axis] >= n)
        if mesh.bc[axis]:
            q[:, axis] %= n
            out[:] = False
        val = np.full(pot.size, np.nan)
        todo = ~out
        # a leaf cell of the same or a coarser depth contains the cube
        for up in range(0, int(dep.max()) + 1):
            if not todo.any():
                break
            dd = dep[todo] - up
            ok = dd >= 0
            idx = np.nonzero(todo)[0][ok]
            k = _key(dd[ok], q[idx] >> up)
            p = np.searchsorted(sorted_keys, k)
            p = np.minimum(p, sorted_keys.size - 1)
            hit = sorted_keys[p] == k
            val[idx[hit]] = pot[order[p[hit]]]
            todo[idx[hit]] = False
        # otherwise finer leaf cells fill the cube: their volume-weighted mean
        for i in np.nonzero(todo)[0]:
            u, s, v = anc[int(dep[i])]
            k = _key(dep[i], q[i])
            p = np.searchsorted(u, k)
            assert p < u.size and u[p] == k
            val[i] = s[p] / v[p]
        return val, ~out

    acc = np.zeros((pot.size, 3))
    for axis in range(3):
        gm, hm = guard(-1, axis)
        gp, hp = guard(+1, axis)
        g2m, _ = guard(-2, axis)
        g2p, _ = guard(+2, axis)
        both = hm & hp
        d = np.where(both, (gp - gm) / (2 * dx[:, axis]), 0.0)
        lo_edge = ~hm & hp
        d = np.where(lo_edge, (-3 * pot + 4 * gp - g2p) / (2 * dx[:, axis]), d)
        hi_edge = hm & ~hp
        d = np.where(hi_edge, -(-3 * pot + 4 * gm - g2m) / (2 * dx[:, axis]), d)
        acc[:, axis] = -d
    return acc
