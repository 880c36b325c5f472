"""GPU path vs the oracle (C-ABI calls through the ctypes binding)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from gpu_util import ensure_library, fso_pack, golden  # noqa: E402
from oracle import basis as ob_basis, ctmrg as octmrg, doublelayer as dl, observables as ob  # noqa: E402
from paper_2410_11596_gb300 import _lib as L, inputs  # noqa: E402
from pins import onsager_log_z, onsager_nn  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    ensure_library()
    from paper_2410_11596_gb300.api import Context
    c = Context(0)
    yield c
    c.close()


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


@pytest.mark.parametrize("D", [1, 2, 3])
@pytest.mark.parametrize("cplx", [False, True])
def test_double_layer_dense(ctx, D, cplx):
    A = inputs.random_ipeps(2, D, 21, complex_valued=cplx)
    q = D * D
    Ad = _dev(A.view(np.float64) if cplx else A)
    out = torch.empty(q ** 4 * (2 if cplx else 1), dtype=torch.float64, device="cuda")
    L.hs_make_double_layer(ctx.handle, Ad, 2, D, L.HS_C128 if cplx else L.HS_F64, out)
    got = out.cpu().numpy()
    if cplx:
        got = got.view(np.complex128)
    np.testing.assert_allclose(got.reshape((q,) * 4), dl.double_layer(A), rtol=0, atol=1e-14)


@pytest.mark.parametrize("D", [1, 2, 3, 4])
@pytest.mark.parametrize("herm", [False, True])
def test_double_layer_blocks(ctx, D, herm):
    A = inputs.random_ipeps(2, D, 22)
    a = dl.double_layer(A)
    if herm:
        at = dl.to_hermitian_basis(a, D)
        s = ob_basis.sector_dims(D)
    else:
        at, s = a, (D * D, 0)
    want = fso_pack(at, [s, s], [s, s])
    buf = torch.empty(L.hs_z2_tensor_bytes(D, int(herm)) // 8, dtype=torch.float64, device="cuda")
    t = L.hs_double_layer_hermitian(ctx.handle, _dev(A), 2, D, L.HS_F64, int(herm), buf)
    assert (t.n_even, t.n_odd) == s
    np.testing.assert_allclose(buf.cpu().numpy(), want, rtol=0, atol=1e-14)


def test_to_hermitian_basis_and_rejection(ctx):
    D = 3
    A = inputs.random_ipeps(2, D, 23)
    a = dl.double_layer(A)
    s = ob_basis.sector_dims(D)
    buf = torch.empty(L.hs_z2_tensor_bytes(D, 1) // 8, dtype=torch.float64, device="cuda")
    L.hs_to_hermitian_basis(ctx.handle, _dev(a), D, L.HS_F64, 1e-13, buf)
    np.testing.assert_allclose(buf.cpu().numpy(), fso_pack(dl.to_hermitian_basis(a, D), [s, s], [s, s]),
                               atol=1e-14)
    # a tensor that is not swap-symmetric has odd blocks and must be refused
    rng = np.random.default_rng(0)
    bad = a + 1e-3 * rng.standard_normal(a.shape)
    with pytest.raises(L.HsError) as e:
        L.hs_to_hermitian_basis(ctx.handle, _dev(bad), D, L.HS_F64, 1e-13, buf)
    assert e.value.status == -4


def _run(ctx, A, chi, moves, basis="hermitian", backend="own", precision="f64", eig="f64"):
    from paper_2410_11596_gb300.api import CTMRG
    c = CTMRG(ctx, A, chi, basis=basis, backend=backend, precision=precision, eig=eig)
    c.run(moves)
    return c


@pytest.mark.parametrize("k", [1, 2])
@pytest.mark.parametrize("basis,backend", [("hermitian", "own"), ("dense", "own"), ("dense", "cublas"),
                                           ("hermitian", "cublas")])
def test_ctmrg_matches_oracle(ctx, k, basis, backend):
    """Gauge-invariant results vs the FP64 oracle at every stored checkpoint, 1e-10 (Sec. II.A)."""
    g = golden(k)
    A = inputs.workload_tensor(k)
    from paper_2410_11596_gb300.api import CTMRG
    c = CTMRG(ctx, A, g["chi"], basis=basis, backend=backend)
    h = inputs.heisenberg_bond()
    done = 0
    for m_str, snap in sorted(g["checkpoints"].items(), key=lambda kv: int(kv[0])):
        m = int(m_str)
        c.run(m - done)
        done = m
        rho, t0, t1 = c.rdm2(h)
        assert t1 / t0 == pytest.approx(snap["energy"], rel=1e-10, abs=1e-12), m
        np.testing.assert_allclose(rho.cpu().numpy() / t0, np.array(snap["rho_re"]), atol=1e-10)
        spec = c.corner_spectrum().cpu().numpy()            # hs_corner_spectrum, on the GPU
        np.testing.assert_allclose(spec, np.array(snap["corner_spectrum"]), atol=1e-10)
    gaps = [x for x in g["gaps"] if x is not None]
    assert min(gaps) > 1e-9   # the seed has no near-degenerate cut


def test_z2_path_is_hermitian_by_construction(ctx):
    """S_err = 0 and rho = rho^T exactly in the Hermitian basis (Sec. III.A, Eq. (4))."""
    A = inputs.workload_tensor(2)
    c = _run(ctx, A, 32, 12)
    eps = c.one_site_env().cpu().numpy()
    assert ob.symmetry_error(eps, 4) < 1e-14
    rho, _, _ = c.rdm2(inputs.heisenberg_bond())
    r = rho.cpu().numpy()
    assert np.array_equal(r, r.T)
    # dense path: rho symmetric only up to rounding
    cd = _run(ctx, A, 32, 12, basis="dense")
    eps_d = cd.one_site_env().cpu().numpy()
    assert ob.symmetry_error(eps_d, 4) < 1e-10


def test_one_site_env_matches_oracle(ctx):
    A = inputs.workload_tensor(1)
    c = _run(ctx, A, 16, 6)
    r = octmrg.run(dl.double_layer(A), 16, 6)
    e_gpu = c.one_site_env().cpu().numpy()
    e_or = ob.one_site_environment(r.C, r.T)
    # gauge invariant: eps itself (all boundary legs are contracted)
    np.testing.assert_allclose(e_gpu / np.abs(e_gpu).max(), e_or / np.abs(e_or).max(), atol=1e-11)


@pytest.mark.parametrize("D", [1, 4])
def test_product_state(ctx, D):
    phi = np.array([0.6, 0.8])
    A = inputs.product_state_ipeps(phi, D)
    c = _run(ctx, A, 8, 3)
    E = c.energy(inputs.heisenberg_bond())
    sx = 2 * 0.6 * 0.8 * 0.5
    sz = (0.36 - 0.64) * 0.5
    assert E == pytest.approx(sx * sx + sz * sz, abs=1e-13)


@pytest.mark.parametrize("beta", [0.3, 0.6])
def test_ising_bond_correlation(ctx, beta):
    A = inputs.ising_ipeps(beta)
    c = _run(ctx, A, 32, 120)
    assert c.energy(inputs.sz_sz_bond()) == pytest.approx(onsager_nn(beta), abs=1e-9)
    # free energy from the oracle's formula applied to the GPU environment
    C, T = c.dense_env()
    lk = ob.log_kappa(C.cpu().numpy(), T.cpu().numpy(), dl.double_layer(A)).real
    assert lk == pytest.approx(onsager_log_z(beta), abs=1e-9)


def test_sector_sizes_sum_and_odd_fraction(ctx):
    A = inputs.workload_tensor(2)
    c = _run(ctx, A, 64, 8)
    qe, qo = 10, 6
    for prev, info in zip(c.infos, c.infos[1:]):
        assert info["chi_even"] + info["chi_odd"] == 64
        assert info["n_even"] == prev["chi_even"] * qe + prev["chi_odd"] * qo
        assert info["n_odd"] == prev["chi_even"] * qo + prev["chi_odd"] * qe
    frac = c.infos[-1]["chi_odd"] / 64
    assert 0.2 < frac < 0.8


@pytest.mark.parametrize("basis", ["hermitian", "dense"])
def test_one_site_rdm_matches_oracle(ctx, basis):
    """HS_RDM_ONE_SITE: rho1 from eps and A, normalised, against the oracle; Tr(rho1 S^z)."""
    A = inputs.workload_tensor(1)
    c = _run(ctx, A, 16, 6, basis=basis)
    r = octmrg.run(dl.double_layer(A), 16, 6)
    sz = np.diag([0.5, -0.5])
    rho, t0, t1 = c.rdm1(sz)
    ref = ob.one_site_rdm(r.C, r.T, A)
    np.testing.assert_allclose(rho.cpu().numpy() / t0, ref / np.trace(ref), atol=1e-11)
    assert t1 / t0 == pytest.approx(np.trace(ref @ sz) / np.trace(ref), abs=1e-11)


@pytest.mark.parametrize("D", [1, 2, 3, 4])
def test_from_hermitian_basis_inverts_the_rotation(ctx, D):
    """hs_from_hermitian_basis(a~) = a, the oracle's dense double layer (Sec. II.B: U orthogonal)."""
    from paper_2410_11596_gb300.api import CTMRG
    A = inputs.random_ipeps(2, D, 41)
    c = CTMRG(ctx, A, max(4, D * D))
    a = c.double_layer_dense().cpu().numpy()
    want = dl.double_layer(A)
    np.testing.assert_allclose(a, want, rtol=0, atol=1e-14 * np.abs(want).max())


def test_corner_spectrum_on_gpu_of_a_projected_corner(ctx):
    """With the FP32-projected eigensolver the new corner is P^T C' P (not diagonal): the GPU
    spectrum equals the oracle's formula applied to the same corner."""
    A = inputs.workload_tensor(2)
    c = _run(ctx, A, 64, 10, eig="f32p")
    C, _ = c.dense_env()
    np.testing.assert_allclose(c.corner_spectrum().cpu().numpy(), ob.corner_spectrum(C.cpu().numpy()), atol=1e-13)
