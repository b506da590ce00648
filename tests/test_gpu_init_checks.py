"""The library's own hydrostatic start and its flow-speed check, through the
C-ABI.

The paper starts its gravity cases (sections "Gravity wave", "Rising bubble",
"Drop impact") from the pressure of the fluid at rest.  With
pfl_params.hydrostatic = 1 and no p0, pfl_init integrates dp/ds = rho(phi) g
along the gravity axis itself; the result must equal the same integration done
by the caller (workloads.column_hydrostatic_pstar) and passed as p0.  pfl_diag
reports a run whose flow speed exceeds PFL_SPEED_LIMIT as unstable.
"""
import numpy as np
import pytest

from paper_2206_11637_gb300 import _lib as L
from paper_2206_11637_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2206_11637_gb300 import build
    build.build_library()


def _sim(p, phi0, u0=None, p0=None, precision="fp64"):
    from paper_2206_11637_gb300.pflbm import Simulation
    return Simulation(p, phi0, u0, p0, precision=precision)


@pytest.mark.parametrize("case", ["gravity_wave", "bubble"])
def test_library_hydrostatic_start_equals_caller_integration(case):
    if case == "gravity_wave":
        p, phi0, _, p0 = W.gravity_wave(50)
        level = 25.0 - 0.5
    else:
        p, phi0, _, _ = W.rising_bubble(24, 40, 20, D=10.0, xi=4.0, M=0.05, hydrostatic=False)
        level = 15.0
        p0 = W.column_hydrostatic_pstar(p, phi0, level)
    a = _sim(p, phi0, None, p0)
    p.hydrostatic, p.p_level = 1, level
    b = _sim(p, phi0, None, None)
    ha, ga = a.populations()
    hb, gb = b.populations()
    assert np.array_equal(ha, hb)
    assert np.abs(gb - ga).max() <= 1e-14 * np.abs(ga).max()
    a.step(20)
    b.step(20)
    fa, fb = a.fields(), b.fields()
    for x, y in zip(fa, fb):
        assert np.abs(x - y).max() <= 1e-13 * max(np.abs(x).max(), 1e-300)


def test_library_hydrostatic_start_along_z_from_device_phi():
    """Gravity along +z: the library integrates along z; the caller's
    integration along y of the transposed lattice is the reference.  phi0 is
    handed over as a device tensor."""
    p, phi0, _, _ = W.rising_bubble(20, 16, 28, D=8.0, xi=4.0, M=0.05, hydrostatic=False)
    g = abs(p.gravity[1])
    # the same set-up with y and z exchanged: gravity along +z
    q = W.Params(p.nx, p.nz, p.ny, p.bc, p.rho_h, p.rho_l, p.nu_h, p.nu_l, p.sigma, p.mobility, p.xi,
                 (0.0, 0.0, g))
    phi_q = np.ascontiguousarray(np.swapaxes(phi0, 0, 1))      # (nz', ny', nx) = (ny, nz, nx)
    # reference: integrate along y of the original layout with gravity -g, then
    # flip sign (gravity +g) and swap the axes back
    p_ref = W.Params(p.nx, p.ny, p.nz, p.bc, p.rho_h, p.rho_l, p.nu_h, p.nu_l, p.sigma, p.mobility, p.xi,
                     (0.0, g, 0.0))
    level = 9.25
    ref = np.ascontiguousarray(np.swapaxes(_column_pstar_signed(p_ref, np.ascontiguousarray(np.swapaxes(phi_q, 0, 1)),
                                                                level), 0, 1))
    a = _sim(q, phi_q, None, ref)
    q.hydrostatic, q.p_level = 1, level
    b = _sim(q, torch.from_numpy(phi_q.reshape(-1).copy()).cuda(), None, None)
    ha, ga = a.populations()
    hb, gb = b.populations()
    assert np.array_equal(ha, hb)
    assert np.abs(gb - ga).max() <= 1e-14 * np.abs(ga).max()


def _column_pstar_signed(p, phi0, level):
    """workloads.column_hydrostatic_pstar for gravity of either sign along y."""
    gy = p.gravity[1]
    rho = p.rho_l + phi0 * (p.rho_h - p.rho_l)
    steps = 0.5 * (rho[:, 1:, :] + rho[:, :-1, :])
    P = np.concatenate([np.zeros_like(rho[:, :1, :]), gy * np.cumsum(steps, axis=1)], axis=1)
    j = min(max(int(np.floor(level)), 0), p.ny - 2)
    t = level - j
    P -= (1.0 - t) * P[:, j:j + 1, :] + t * P[:, j + 1:j + 2, :]
    return 3.0 * P / rho


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16s"])
def test_speed_limit_flags_fast_flow(precision):
    p = W.Params(16, 12, 10, (0,) * 6, 1.0, 1e-3, 1 / 60, 1 / 60, 1e-4, 0.02, 4.0)
    phi0 = np.ones(p.shape)
    for speed, ok in ((0.1, True), (0.35, False)):
        u0 = np.zeros((3,) + p.shape)
        u0[0] = speed
        s = _sim(p, phi0, u0, None, precision)
        tol = {"fp64": 1e-14, "fp32": 1e-6, "fp16s": 2e-3}[precision]
        assert abs(s.max_speed() - speed) <= tol * speed
        out, nf = s.diag(check=False)
        st = s.lib.pfl_diag(s.ctx, None, None)
        assert nf == 0
        if ok:
            assert st == L.PFL_OK
        else:
            assert st == L.PFL_ERR_UNSTABLE
            assert "flow speed" in s.lib.pfl_last_error().decode()
