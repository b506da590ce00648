"""The C-ABI library loads and exports every declared symbol; host-side
argument checks (no GPU needed)."""
import ctypes

import pytest

from paper_2206_11637_gb300 import _lib as L
from paper_2206_11637_gb300 import build as B
from paper_2206_11637_gb300 import workloads as W
from paper_2206_11637_gb300 import pflbm


@pytest.fixture(scope="module")
def lib():
    B.build_library()
    return L.load()


def test_exports_every_declared_symbol(lib):
    names = L.declared_symbols()
    assert {"pfl_init", "pfl_step", "pfl_fields", "pfl_diag"} <= set(names)
    for n in names:
        assert hasattr(lib, n), n
    assert lib.pfl_version() == 3


def test_workspace_size(lib):
    p, _, _, _ = W.static_drop(16, 5.0)
    n = p.cells
    b64 = pflbm.workspace_bytes(p, L.PFL_FP64)
    b32 = pflbm.workspace_bytes(p, L.PFL_FP32)
    b16 = pflbm.workspace_bytes(p, L.PFL_FP16S)
    assert b64 >= 42 * n * 8 + n * 8
    assert b32 >= 42 * n * 4 + n * 4
    assert b16 >= 42 * n * 2 + n * 4
    assert b16 < b32 < b64


def test_workspace_grows_with_the_phase_field_lattice(lib):
    p, _, _, _ = W.static_drop(16, 5.0)
    n = p.cells
    for prec, s in ((L.PFL_FP64, 8), (L.PFL_FP32, 4), (L.PFL_FP16S, 2)):
        b15 = pflbm.workspace_bytes(p, prec)
        p.h_lattice = 27
        b27 = pflbm.workspace_bytes(p, prec)
        p.h_lattice = 15
        # two array pairs (fused engine): 2 x 12 more h populations per cell
        assert b27 - b15 >= 2 * 12 * n * s
        assert b27 - b15 < 2 * 12 * n * s + 4096


@pytest.mark.parametrize("field,value", [("mobility", 0.0), ("xi", -1.0), ("rho_l", 0.0), ("nu_h", -0.2),
                                         ("nu_l", -0.1), ("nx", 0), ("h_lattice", 19),
                                         ("h_lattice", 9)])   # 9 (D2Q9) needs nz = 1
def test_rejects_bad_parameters(lib, field, value):
    p, phi0, _, _ = W.static_drop(8, 3.0)
    setattr(p, field, value)
    s = pflbm._params_struct(p, 0)
    assert lib.pfl_workspace_bytes(ctypes.byref(s)) == 0
    ctx = ctypes.c_void_p()
    st = lib.pfl_init(ctypes.byref(s), None, None, None, None, 0, None, ctypes.byref(ctx))
    assert st == L.PFL_ERR_ARG
    assert lib.pfl_last_error().decode() != ""


def test_rejects_mixed_faces(lib):
    p, _, _, _ = W.static_drop(8, 3.0)
    p.bc = (0, 1, 0, 0, 0, 0)
    s = pflbm._params_struct(p, 0)
    assert lib.pfl_workspace_bytes(ctypes.byref(s)) == 0


def test_null_context_calls(lib):
    assert lib.pfl_step(None, 1) == L.PFL_ERR_ARG
    assert lib.pfl_fields(None, None, None, None, None) == L.PFL_ERR_ARG
    assert lib.pfl_time(None) == -1
    assert lib.pfl_set_graph_steps(None, 2) == L.PFL_ERR_ARG
    assert lib.pfl_state_bytes(None) == 0
    assert lib.pfl_save(None, None, 0) == L.PFL_ERR_ARG
    assert lib.pfl_load(None, None, 0) == L.PFL_ERR_ARG
    assert lib.pfl_interface_height(None, 0, 0, None) == L.PFL_ERR_ARG
    lib.pfl_destroy(None)


def test_batch_takes_d3q15_instances_only(lib):
    p, _, _, _ = W.static_drop(16, 5.0)
    arr = (L.pfl_params * 1)(pflbm._params_struct(p, L.PFL_FP32))
    assert lib.pfl_batch_workspace_bytes(arr, 1) > 0
    p.h_lattice = 27
    arr = (L.pfl_params * 1)(pflbm._params_struct(p, L.PFL_FP32))
    assert lib.pfl_batch_workspace_bytes(arr, 1) == 0


def test_two_d_lattice_workspace(lib):
    p, _, _, _ = W.capillary_wave(32, ny=32)
    n = p.cells
    b3 = pflbm.workspace_bytes(p, L.PFL_FP32)
    p.h_lattice = 9
    b2 = pflbm.workspace_bytes(p, L.PFL_FP32)
    # two array pairs of (9 + 9) instead of (15 + 27) populations per cell
    assert b3 - b2 >= 2 * 24 * n * 4


def test_hydrostatic_start_needs_gravity_along_one_axis(lib):
    p, _, _, _ = W.rising_bubble(16, 24, 16, D=8.0)
    p.hydrostatic, p.p_level = 1, 12.0
    assert pflbm.workspace_bytes(p, L.PFL_FP32) > 0
    p.gravity = (1e-6, -1e-6, 0.0)
    assert pflbm.workspace_bytes(p, L.PFL_FP32) == 0
    p.gravity = (0.0, 0.0, 0.0)
    assert pflbm.workspace_bytes(p, L.PFL_FP32) == 0
    p.gravity, p.p_level = (0.0, -1e-6, 0.0), float("nan")
    assert pflbm.workspace_bytes(p, L.PFL_FP32) == 0
    p.hydrostatic = 2
    assert pflbm.workspace_bytes(p, L.PFL_FP32) == 0


def test_null_context_speed(lib):
    assert lib.pfl_max_speed(None, None) == L.PFL_ERR_ARG


def test_host_hydrostatic_start(lib):
    """pfl_hydrostatic_pstar (host only): equal to the caller-side column
    integration for gravity along -y; gravity along z gives the y result of
    the transposed field (the integration follows the gravity axis, whichever
    it is); the refusals."""
    import numpy as np
    p, phi0, _, _ = W.gravity_wave(24)
    p.p_level = 11.5
    ours = pflbm.hydrostatic_pstar(p, phi0)
    ref = W.column_hydrostatic_pstar(p, phi0, 11.5)
    assert np.allclose(ours, ref, rtol=1e-13, atol=1e-15)

    p3, _, _, _ = W.rising_bubble(12, 20, 8, D=5.0, hydrostatic=False)
    rng = np.random.Generator(np.random.PCG64(3))
    phi = rng.uniform(0.0, 1.0, p3.shape)                  # (nz, ny, nx)
    p3.gravity, p3.p_level = (0.0, -2e-5, 0.0), 7.25
    along_y = pflbm.hydrostatic_pstar(p3, phi)
    pz = W.Params(p3.nx, p3.nz, p3.ny, p3.bc, p3.rho_h, p3.rho_l, p3.nu_h, p3.nu_l, p3.sigma, p3.mobility, p3.xi,
                  (0.0, 0.0, -2e-5))                       # y and z swapped
    pz.p_level = 7.25
    along_z = pflbm.hydrostatic_pstar(pz, np.ascontiguousarray(phi.transpose(1, 0, 2)))
    assert np.array_equal(along_z.transpose(1, 0, 2), along_y)
    # flipping gravity flips the pressure
    p3.gravity = (0.0, 2e-5, 0.0)
    assert np.allclose(pflbm.hydrostatic_pstar(p3, phi), -along_y, rtol=1e-14, atol=0)

    out = np.empty(p3.shape)
    s = pflbm._params_struct(p3, 0)
    assert lib.pfl_hydrostatic_pstar(ctypes.byref(s), None, out.ctypes.data_as(ctypes.c_void_p)) == L.PFL_ERR_ARG
    p3.gravity = (1e-6, 1e-6, 0.0)
    s = pflbm._params_struct(p3, 0)
    assert lib.pfl_hydrostatic_pstar(ctypes.byref(s), phi.ctypes.data_as(ctypes.c_void_p),
                                     out.ctypes.data_as(ctypes.c_void_p)) == L.PFL_ERR_ARG
    assert "one axis" in lib.pfl_last_error().decode()
