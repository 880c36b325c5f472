"""Directional CTMRG (no lattice symmetry) on the GPU against the oracle: kept singular values of
every move, one-site and both two-site reduced density matrices and the free energy per site,
computed from the GPU's environment and from the oracle's, on seeded tensors with no symmetry."""
import numpy as np
import pytest
import torch

from oracle import ctmrg_directional as cd, doublelayer as dl, observables as ob
from paper_2410_11596_gb300 import inputs
from pins import onsager_log_z_aniso, onsager_nn_aniso

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2410_11596_gb300.api import Context
    c = Context(0)
    yield c
    c.close()


def _tensor(D, seed):
    return inputs.asymmetric_ipeps(2, D, inputs.SEED_BASE + 5100 + seed)


def _gpu_env(c):
    return [x.cpu().numpy() for x in c.dense_env()]


def _observables(E, A, a):
    r1 = cd.one_site_rdm(E, A)
    rh = cd.two_site_rdm_horizontal(E, A)
    rv = cd.two_site_rdm_vertical(E, A)
    return r1 / np.trace(r1), rh / np.trace(rh), rv / np.trace(rv), cd.log_kappa(E, a)


def _compare(c, r, A, a, tol):
    go = _observables(_gpu_env(c), A, a)
    oo = _observables(r.E, A, a)
    errs = [float(np.abs(x - y).max()) for x, y in zip(go[:3], oo[:3])] + [abs(go[3] - oo[3])]
    return errs


# (D, chi, sweeps, seed, basis): the smallest case, truncation from the first move (chi < q),
# ragged sectors (q = 9 = 6 + 3), several GEMM tiles per block (chi q = 1024), the plain basis
CASES = [(2, 16, 20, 1, "hermitian"), (2, 3, 6, 3, "hermitian"), (3, 27, 10, 2, "hermitian"),
         (4, 64, 5, 4, "hermitian"), (2, 16, 20, 1, "dense"), (3, 27, 6, 2, "dense")]


@pytest.mark.parametrize("D,chi,sweeps,seed,basis", CASES)
def test_directional_ctmrg_matches_oracle(ctx, D, chi, sweeps, seed, basis):
    """FP64 GEMMs and FP64 SVD on both sides.

    Jacobi SVD: kept singular values (divided by the largest) of every move within 1e-12; rho
    (one site, horizontal and vertical pairs, trace-normalised) and ln kappa after the last sweep
    within 1e-10, the FP64 gate. The projectors carry S^-1/2 with kept s down to 1e-7..1e-12 of
    the largest, so the environment itself agrees only in the gauge-invariant quantities."""
    from paper_2410_11596_gb300.api import DirectionalCTMRG
    A = _tensor(D, seed)
    a = dl.double_layer(A)
    r = cd.run(a, chi, sweeps)
    assert r.min_gap > 1e-8
    c = DirectionalCTMRG(ctx, A, chi, basis=basis)
    c.run(sweeps)
    assert len(c.infos) == len(r.infos) == 4 * sweeps
    worst = 0.0
    for k, (gi, oi, sv) in enumerate(zip(c.infos, r.infos, c.spectra)):
        assert len(sv) == len(oi.kept), k
        worst = max(worst, float(np.abs(np.array(sv) - oi.kept).max()))
        assert gi["direction"] == k % 4
    print(f"D={D} chi={chi} {basis}: max |d s/s_max| over {len(c.infos)} moves = {worst:.2e}")
    assert worst <= 1e-12
    errs = _compare(c, r, A, a, 1e-10)
    print(f"  |d rho1|, |d rho_h|, |d rho_v|, |d ln kappa| = " + ", ".join(f"{e:.2e}" for e in errs))
    assert max(errs) <= 1e-10
    if basis == "hermitian" and D > 1:
        qe, qo = D * (D + 1) // 2, D * (D - 1) // 2
        assert (c.env.q_even, c.env.q_odd) == (qe, qo)
        if chi >= D * D:       # both sectors populated on every bond (at chi = 3 all three are even)
            for b in range(4):
                assert c.env.chi_even[b] > 0 and c.env.chi_odd[b] > 0


@pytest.mark.parametrize("D,chi,sweeps,seed,basis", [CASES[2], CASES[3], CASES[5]])
def test_polar_svd_mode_matches_oracle(ctx, D, chi, sweeps, seed, basis):
    """The polar-decomposition SVD (the faster mode): rho and ln kappa within the FP64 gate 1e-10;
    its kept singular values within 1e-8 of the largest (measured up to 1.7e-9: a backward-stable
    SVD whose singular values carry absolute errors of order 1e-11..1e-9 of the largest, against
    1e-14 for the Jacobi SVD)."""
    from paper_2410_11596_gb300.api import DirectionalCTMRG
    A = _tensor(D, seed)
    a = dl.double_layer(A)
    r = cd.run(a, chi, sweeps)
    c = DirectionalCTMRG(ctx, A, chi, basis=basis, svd="polar")
    c.run(sweeps)
    worst = max(float(np.abs(np.array(sv) - oi.kept).max()) for oi, sv in zip(r.infos, c.spectra))
    errs = _compare(c, r, A, a, 1e-10)
    print(f"polar D={D} chi={chi} {basis}: s {worst:.2e}, rho/ln kappa " + ", ".join(f"{e:.2e}" for e in errs))
    assert worst <= 1e-8
    assert max(errs) <= 1e-10


def test_sector_sizes_follow_the_kept_spectrum(ctx):
    """The kept sectors of each bond are the parity counts of the chi largest singular values;
    their sum is the bond dimension and no bond exceeds chi."""
    from paper_2410_11596_gb300.api import DirectionalCTMRG
    c = DirectionalCTMRG(ctx, _tensor(3, 2), 20, basis="hermitian")
    c.run(3)
    for info in c.infos:
        assert info["chi_even"] + info["chi_odd"] <= 20
        assert info["s_cut"] <= info["s_max"] and info["s_next"] <= info["s_cut"]
    for b in range(4):
        assert c.bond(b) <= 20


@pytest.mark.parametrize("bx,by", [(0.3, 0.5), (0.5, 0.7)])
def test_anisotropic_ising_matches_onsager(ctx, bx, by):
    """The GPU environment of the anisotropic Ising network: free energy per site and the
    bond correlations along x and y from Onsager's solution."""
    from paper_2410_11596_gb300.api import DirectionalCTMRG
    A = inputs.anisotropic_ising_ipeps(bx, by)
    a = dl.double_layer(A)
    c = DirectionalCTMRG(ctx, A, 24, basis="hermitian")
    c.run(60)
    E = _gpu_env(c)
    zz = inputs.sz_sz_bond()
    assert cd.log_kappa(E, a) == pytest.approx(onsager_log_z_aniso(bx, by), abs=1e-10)
    assert ob.bond_energy(cd.two_site_rdm_horizontal(E, A), zz) == pytest.approx(onsager_nn_aniso(bx, by), abs=1e-9)
    assert ob.bond_energy(cd.two_site_rdm_vertical(E, A), zz) == pytest.approx(onsager_nn_aniso(by, bx), abs=1e-9)


def test_product_state_closed_form(ctx):
    """D = 1 (one even state per leg, no odd sector): every bond stays one-dimensional and the
    one-site RDM is |phi><phi| / <phi|phi>."""
    from paper_2410_11596_gb300.api import DirectionalCTMRG
    phi = np.array([0.6, -0.8])
    A = inputs.product_state_ipeps(phi, 1).real.copy()
    c = DirectionalCTMRG(ctx, A, 4, basis="hermitian")
    c.run(2)
    assert all(c.bond(b) == 1 for b in range(4))
    r1 = cd.one_site_rdm(_gpu_env(c), A)
    np.testing.assert_allclose(r1 / np.trace(r1), np.outer(phi, phi) / phi.dot(phi), atol=1e-14)


def test_c4v_input_agrees_with_the_c4v_path(ctx):
    """A C4v tensor: the directional GPU run and the C4v GPU run approximate the same network;
    their bond energies agree at the truncation level (1e-7 at D = 2, chi = 16) and the
    horizontal and vertical bonds agree with each other."""
    from paper_2410_11596_gb300.api import CTMRG, DirectionalCTMRG
    A = inputs.random_ipeps(2, 2, inputs.SEED_BASE + 1)
    h = inputs.heisenberg_bond()
    c4 = CTMRG(ctx, A, 16, basis="hermitian")
    c4.run(60)
    e4 = c4.energy(h)
    c = DirectionalCTMRG(ctx, A, 16, basis="hermitian")
    c.run(30)
    E = _gpu_env(c)
    eh = ob.bond_energy(cd.two_site_rdm_horizontal(E, A), h)
    ev = ob.bond_energy(cd.two_site_rdm_vertical(E, A), h)
    assert eh == pytest.approx(ev, abs=1e-10)
    assert eh == pytest.approx(e4, abs=1e-7)


def test_bad_arguments_are_reported(ctx):
    from paper_2410_11596_gb300 import _lib as L
    from paper_2410_11596_gb300.api import DirectionalCTMRG
    c = DirectionalCTMRG(ctx, _tensor(2, 1), 8)
    with pytest.raises(L.HsError):
        L.hs_ctmrg4_move(ctx.handle, c.a, c.env, 8, 4)        # no fifth side
    with pytest.raises(L.HsError):
        L.hs_ctmrg4_move(ctx.handle, c.a, c.env, 10 ** 6, 0)  # chi above chi_max
    torch.cuda.synchronize()
