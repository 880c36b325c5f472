"""GPU HOTRG in the Hermitian basis vs the dense FP64 oracle HOTRG and Onsager (Sec. II.A)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from gpu_util import ensure_library  # noqa: E402
from oracle import doublelayer as dl, hotrg as oh  # noqa: E402
from paper_2410_11596_gb300 import inputs  # noqa: E402
from pins import onsager_log_z  # noqa: E402

pytestmark = pytest.mark.gpu

# ln Z per site with TF32x3 block GEMMs: a 3-pass TF32 product is accurate to about
# u = 2^-21 of sum |a_i b_i| (the lo parts are rounded to TF32), i.e. to u kappa relative,
# kappa = sum |a_i b_i| / |sum a_i b_i| <= sqrt(K) for random signs (K <= chi^2 = 256 here:
# kappa <= 16). It enters ln Z through the normalisations ln c_k / 2^k, summing to at most
# twice one step's error: 2 u sqrt(256) = 1.5e-5.
TF32X3_LNZ_TOL = 1.5e-5


@pytest.fixture(scope="module")
def ctx():
    ensure_library()
    from paper_2410_11596_gb300.api import Context
    c = Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("beta", [0.3, 0.6])
def test_ising_log_z(ctx, beta):
    from paper_2410_11596_gb300.api import HOTRG
    A = inputs.ising_ipeps(beta)
    h = HOTRG(ctx, A, 16)
    h.run(30)
    ref = oh.log_z_per_site(oh.run(dl.double_layer(A), 16, 30))
    assert h.log_z_per_site() == pytest.approx(ref, abs=1e-10)
    assert h.log_z_per_site() == pytest.approx(onsager_log_z(beta), abs=2e-9)


@pytest.mark.parametrize("basis", ["hermitian", "dense"])
@pytest.mark.parametrize("chi,steps", [(6, 6), (8, 9)])
def test_random_tensor_matches_oracle(ctx, basis, chi, steps):
    """ln Z per site and the normalised Gram spectra of every step vs the oracle."""
    from paper_2410_11596_gb300.api import HOTRG
    A = inputs.workload_tensor(1)
    h = HOTRG(ctx, A, chi, basis=basis)
    h.run(steps)
    r = oh.run(dl.double_layer(A), chi, steps)
    assert h.log_z_per_site() == pytest.approx(oh.log_z_per_site(r), rel=1e-11, abs=1e-12)
    kept = [i["h_even"] + i["h_odd"] for i in h.infos]
    assert kept == [min(chi, len(w)) for w in r.spectra]
    if basis == "hermitian":
        assert all(i["h_odd"] > 0 for i in h.infos[1:])


def test_sector_bookkeeping(ctx):
    from paper_2410_11596_gb300.api import HOTRG
    h = HOTRG(ctx, inputs.workload_tensor(2), 12)      # D = 4: q = 16 = 10 + 6
    info = h.step()
    assert (h.t.v_even, h.t.v_odd) == (10, 6)           # vertical legs untouched by a vertical step
    assert (h.t.h_even, h.t.h_odd) == (info["h_even"], info["h_odd"])
    assert info["h_even"] + info["h_odd"] == 12
    info = h.step()                                     # horizontal step truncates the vertical legs
    assert (h.t.v_even + h.t.v_odd) == 12


@pytest.mark.parametrize("basis", ["hermitian", "dense"])
@pytest.mark.parametrize("mirror", [False, True])
def test_side_choice_on_lopsided_network(ctx, basis, mirror):
    """A network that is not mirror symmetric: the first step takes the right Gram matrix
    (the left one when the tensor is mirrored), as the oracle does, and ln Z per site after
    four steps matches the oracle."""
    from paper_2410_11596_gb300.api import HOTRG
    A = inputs.lopsided_ipeps()
    if mirror:
        A = np.ascontiguousarray(A.transpose(0, 1, 4, 3, 2))
    h = HOTRG(ctx, A, 4, basis=basis)
    h.run(4)
    r = oh.run(dl.double_layer(A), 4, 4)
    assert [i["side"] for i in h.infos] == r.sides
    assert r.sides[0] == (0 if mirror else 1)
    assert h.infos[0]["discarded_right" if not mirror else "discarded_left"] < \
        h.infos[0]["discarded_left" if not mirror else "discarded_right"]
    assert h.log_z_per_site() == pytest.approx(oh.log_z_per_site(r), rel=1e-10, abs=1e-12)


@pytest.mark.parametrize("basis", ["hermitian", "dense"])
@pytest.mark.parametrize("beta,chi,steps", [(0.3, 16, 30), (0.6, 16, 30)])
def test_tf32x3_ising_log_z(ctx, basis, beta, chi, steps):
    """HOTRG with its block GEMMs on tcgen05 (TF32x3, FP32 accumulation; FP64 Gram eig):
    ln Z per site within TF32X3_LNZ_TOL of the FP64 oracle."""
    from paper_2410_11596_gb300.api import HOTRG
    A = inputs.ising_ipeps(beta)
    h = HOTRG(ctx, A, chi, basis=basis, precision="tf32x3")
    h.run(steps)
    ref = oh.log_z_per_site(oh.run(dl.double_layer(A), chi, steps))
    print(f"tf32x3 HOTRG beta={beta} {basis}: |d lnZ| = {abs(h.log_z_per_site() - ref):.2e}")
    assert h.log_z_per_site() == pytest.approx(ref, abs=TF32X3_LNZ_TOL)


@pytest.mark.parametrize("chi,steps", [(8, 9), (16, 6)])
def test_tf32x3_random_tensor(ctx, chi, steps):
    """Random real tensor (workload 1), TF32x3 GEMMs in the Hermitian basis: ln Z per site
    within TF32X3_LNZ_TOL of the oracle and the same number of kept states per step."""
    from paper_2410_11596_gb300.api import HOTRG
    A = inputs.workload_tensor(1)
    h = HOTRG(ctx, A, chi, precision="tf32x3")
    h.run(steps)
    r = oh.run(dl.double_layer(A), chi, steps)
    print(f"tf32x3 HOTRG chi={chi}: |d lnZ| = {abs(h.log_z_per_site() - oh.log_z_per_site(r)):.2e}")
    assert h.log_z_per_site() == pytest.approx(oh.log_z_per_site(r), abs=TF32X3_LNZ_TOL)
    assert [i["h_even"] + i["h_odd"] for i in h.infos] == [min(chi, len(w)) for w in r.spectra]
