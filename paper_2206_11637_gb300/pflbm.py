"""Python front end of the PFLBM library.

``Simulation`` owns one context of libpflbm.so.  PyTorch provides the device
workspace (a uint8 tensor) and the CUDA stream; every computation runs in the
library's kernels.
"""
import ctypes

import numpy as np

from . import _lib as L


def _params_struct(p, precision):
    s = L.pfl_params()
    s.nx, s.ny, s.nz = int(p.nx), int(p.ny), int(p.nz)
    for k in range(6):
        s.bc[k] = int(p.bc[k])
    s.rho_h, s.rho_l = float(p.rho_h), float(p.rho_l)
    s.nu_h, s.nu_l = float(p.nu_h), float(p.nu_l)
    s.sigma, s.mobility, s.xi = float(p.sigma), float(p.mobility), float(p.xi)
    for k in range(3):
        s.gravity[k] = float(p.gravity[k])
    s.precision = int(precision)
    s.collision = int(p.collision)
    s.engine = int(getattr(p, "engine", 0))
    s.h_lattice = int(getattr(p, "h_lattice", 15))
    s.solids = 1 if getattr(p, "solid", None) is not None else 0
    s.hydrostatic = int(getattr(p, "hydrostatic", 0))
    s.p_level = float(getattr(p, "p_level", 0.0))
    return s


def _ptr(a):
    """Data pointer of a numpy array or a torch tensor (None passes NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data_as(ctypes.c_void_p)
    return ctypes.c_void_p(a.data_ptr())


def workspace_bytes(p, precision):
    s = _params_struct(p, precision)
    return L.load().pfl_workspace_bytes(ctypes.byref(s))


def hydrostatic_pstar(p, phi0):
    """The library's hydrostatic start (pfl_hydrostatic_pstar, on the host):
    p* of the fluid at rest under p.gravity, zero pressure at p.p_level along
    the gravity axis; phi0 and the result are (nz, ny, nx) FP64 arrays."""
    s = _params_struct(p, L.PFL_FP64)
    phi0 = np.ascontiguousarray(np.asarray(phi0, dtype=np.float64))
    if phi0.size != p.nx * p.ny * p.nz:
        raise ValueError("phi0 must hold one value per cell")
    out = np.empty((p.nz, p.ny, p.nx))
    L.check(L.load().pfl_hydrostatic_pstar(ctypes.byref(s), _ptr(phi0), _ptr(out)))
    return out


class Simulation:
    """One PFLBM domain on the GPU.

    p: a ``workloads.Params``-like object; phi0 (N), u0 (3N SoA) and p0 (N)
    are FP64 host arrays or CUDA tensors (u0, p0 optional).
    """

    PRECISIONS = {"fp64": L.PFL_FP64, "fp32": L.PFL_FP32, "fp16s": L.PFL_FP16S}

    def __init__(self, p, phi0, u0=None, p0=None, precision="fp64", device=None, stream=None):
        import torch
        self.lib = L.load()
        self.torch = torch
        self.p = p
        self.precision = self.PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        self.shape = (p.nz, p.ny, p.nx)
        self.N = p.nx * p.ny * p.nz
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        self._params = _params_struct(p, self.precision)
        nbytes = self.lib.pfl_workspace_bytes(ctypes.byref(self._params))
        if nbytes == 0:
            raise L.PFLError(L.PFL_ERR_ARG, "invalid parameters")
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self.stream = torch.cuda.current_stream(self.device) if stream is None else stream
        inputs = [self._as_f64(a, n) for a, n in ((phi0, self.N), (u0, 3 * self.N), (p0, self.N))]
        self._keep = inputs
        ctx = ctypes.c_void_p()
        L.check(self.lib.pfl_init(ctypes.byref(self._params), _ptr(inputs[0]), _ptr(inputs[1]), _ptr(inputs[2]),
                                  ctypes.c_void_p(self.workspace.data_ptr()), nbytes,
                                  ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(ctx)))
        self.ctx = ctx
        self._keep = None
        solid = getattr(p, "solid", None)
        if solid is not None:   # solid cells (nonzero), (nz, ny, nx)
            mask = np.ascontiguousarray(np.asarray(solid).reshape(-1) != 0, dtype=np.uint8)
            if mask.size != self.N:
                raise ValueError("solid mask must hold one byte per cell")
            L.check(self.lib.pfl_set_solid(self.ctx, _ptr(mask)))

    def _as_f64(self, a, n):
        if a is None:
            return None
        torch = self.torch
        if isinstance(a, torch.Tensor):
            a = a.detach().to(torch.float64).contiguous().reshape(-1)
        else:
            a = np.ascontiguousarray(np.asarray(a, dtype=np.float64)).reshape(-1)
        count = a.numel() if hasattr(a, "numel") else a.size
        if count != n:
            raise ValueError("expected %d values, got %d" % (n, count))
        return a

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.pfl_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def time(self):
        return self.lib.pfl_time(self.ctx)

    def step(self, n=1):
        L.check(self.lib.pfl_step(self.ctx, int(n)))

    def interface_height(self, x=0, z=0):
        """First phi = 1/2 crossing along y of the column (x, z), from the
        heavy side, interpolated linearly (pfl_interface_height); NaN if none."""
        y = ctypes.c_double()
        L.check(self.lib.pfl_interface_height(self.ctx, int(x), int(z), ctypes.byref(y)))
        return y.value

    def save(self, out=None):
        """The saved state (pfl_save) as a uint8 array, or into `out` (a host
        uint8 numpy array or a CUDA uint8 tensor of at least state_bytes)."""
        n = int(self.lib.pfl_state_bytes(self.ctx))
        if out is None:
            out = np.empty(n, dtype=np.uint8)
        ptr = out.data_ptr() if hasattr(out, "data_ptr") else out.ctypes.data
        size = out.numel() if hasattr(out, "numel") else out.nbytes
        L.check(self.lib.pfl_save(self.ctx, ctypes.c_void_p(ptr), ctypes.c_size_t(size)))
        return out

    def load(self, state):
        """Resume from a saved state (pfl_load): host array or CUDA tensor."""
        if hasattr(state, "data_ptr"):
            ptr, size = state.data_ptr(), state.numel() * state.element_size()
        else:
            state = np.ascontiguousarray(state, dtype=np.uint8)
            ptr, size = state.ctypes.data, state.nbytes
        L.check(self.lib.pfl_load(self.ctx, ctypes.c_void_p(ptr), ctypes.c_size_t(size)))

    def set_graph_steps(self, k):
        """Steps per replayed CUDA graph of the fused engine (0: none)."""
        L.check(self.lib.pfl_set_graph_steps(self.ctx, int(k)))

    def adjoint(self, n_steps, observations):
        """Discrete adjoint over the next n_steps steps.

        observations: list of (step, W) with W an (N,) FP64 array or CUDA
        tensor; J = sum_o sum_x W_o(x) phi(x, t0 + step_o).  Returns
        (J, [dJ/dM, dJ/dxi, dJ/dsigma]); the simulation advances n_steps.
        """
        torch = self.torch
        nbytes = self.lib.pfl_adjoint_workspace_bytes(self.ctx, int(n_steps))
        if nbytes == 0:
            raise L.PFLError(L.PFL_ERR_ARG, "invalid adjoint request")
        ws = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        steps = (ctypes.c_int * len(observations))(*[int(k) for k, _ in observations])
        keep = [self._as_f64(w, self.N) for _, w in observations]
        ptrs = (ctypes.c_void_p * len(keep))(*[_ptr(w).value for w in keep])
        J = ctypes.c_double(0.0)
        grad = np.zeros(3)
        L.check(self.lib.pfl_adjoint(self.ctx, int(n_steps), len(observations), ctypes.cast(steps, ctypes.c_void_p),
                                     ctypes.cast(ptrs, ctypes.c_void_p), ctypes.c_void_p(ws.data_ptr()), nbytes,
                                     ctypes.byref(J), _ptr(grad)))
        del ws
        return J.value, grad

    def kernel_times(self, n):
        """Run n steps timing each kernel with CUDA events: (ms step kernel, ms phi pass)."""
        ms = np.zeros(2)
        L.check(self.lib.pfl_kernel_times(self.ctx, int(n), _ptr(ms)))
        return float(ms[0]), float(ms[1])

    def fields(self, out=None):
        """phi, rho, p, u as host numpy arrays ((nz,ny,nx) and (3,nz,ny,nx)).

        With ``out`` = dict of CUDA float64 tensors (keys phi, rho, p, u) the
        fields are written there on the device instead.
        """
        if out is not None:
            L.check(self.lib.pfl_fields(self.ctx, _ptr(out.get("phi")), _ptr(out.get("rho")), _ptr(out.get("p")),
                                        _ptr(out.get("u"))))
            return out
        phi = np.empty(self.shape)
        rho = np.empty(self.shape)
        pr = np.empty(self.shape)
        u = np.empty((3,) + self.shape)
        L.check(self.lib.pfl_fields(self.ctx, _ptr(phi), _ptr(rho), _ptr(pr), _ptr(u)))
        return phi, rho, pr, u

    def phi(self):
        phi = np.empty(self.shape)
        L.check(self.lib.pfl_fields(self.ctx, _ptr(phi), None, None, None))
        return phi

    @property
    def qh(self):
        """Velocities of the phase-field lattice (15, 27, or 9 in 2-D)."""
        return {27: 27, 9: 9}.get(self._params.h_lattice, 15)

    @property
    def qg(self):
        """Velocities of the hydrodynamic lattice (27, or 9 in 2-D)."""
        return 9 if self.qh == 9 else 27

    def populations(self):
        h = np.empty((self.qh,) + self.shape)
        g = np.empty((self.qg,) + self.shape)
        L.check(self.lib.pfl_populations(self.ctx, _ptr(h), _ptr(g)))
        return h, g

    def set_populations(self, h, g):
        h = np.ascontiguousarray(h, dtype=np.float64)
        g = np.ascontiguousarray(g, dtype=np.float64)
        if h.size != self.qh * self.N or g.size != self.qg * self.N:
            raise ValueError("populations must hold %d h and %d g values per cell" % (self.qh, self.qg))
        L.check(self.lib.pfl_set_populations(self.ctx, _ptr(h), _ptr(g)))

    def diag(self, check=True):
        """FP64 sums [phi, phi x, phi y, phi z, 1-phi, ...] and the non-finite count."""
        out = np.empty(8)
        nf = ctypes.c_longlong(0)
        st = self.lib.pfl_diag(self.ctx, _ptr(out), ctypes.byref(nf))
        if check:
            L.check(st)
        return out, int(nf.value)

    def max_speed(self):
        """Largest flow speed |u| over the fluid cells (pfl_max_speed)."""
        v = ctypes.c_double(0.0)
        L.check(self.lib.pfl_max_speed(self.ctx, ctypes.byref(v)))
        return v.value

    def mass(self):
        return self.diag()[0][0]
