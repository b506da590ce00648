"""Python front end of the batched PFLBM (pfl_batch_* in include/pflbm.h)."""
import ctypes

import numpy as np

from . import _lib as L
from .pflbm import _params_struct, _ptr, Simulation


class Batch:
    """Independent lattices advanced together by persistent launches.

    instances: list of (params, phi0, u0, p0) with workloads.Params-like params;
    every instance uses `precision`.  tune=True lets the library time the
    candidate launch shapes at init.
    """

    def __init__(self, instances, precision="fp32", tune=True, device=None, stream=None):
        import torch
        self.lib = L.load()
        self.torch = torch
        prec = Simulation.PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        self.count = len(instances)
        self.params = [q for q, _, _, _ in instances]
        arr = (L.pfl_params * self.count)(*[_params_struct(q, prec) for q in self.params])
        self._arr = arr
        nbytes = self.lib.pfl_batch_workspace_bytes(arr, self.count)
        if nbytes == 0:
            raise L.PFLError(L.PFL_ERR_ARG, "invalid batch parameters")
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self.stream = torch.cuda.current_stream(self.device) if stream is None else stream
        keep, phis, us, ps = [], [], [], []
        for q, phi0, u0, p0 in instances:
            n = q.nx * q.ny * q.nz
            a = np.ascontiguousarray(np.asarray(phi0, dtype=np.float64)).reshape(-1)
            assert a.size == n
            keep.append(a)
            phis.append(a.ctypes.data)
            if u0 is not None:
                b = np.ascontiguousarray(np.asarray(u0, dtype=np.float64)).reshape(-1)
                keep.append(b)
                us.append(b.ctypes.data)
            else:
                us.append(None)
            if p0 is not None:
                c = np.ascontiguousarray(np.asarray(p0, dtype=np.float64)).reshape(-1)
                keep.append(c)
                ps.append(c.ctypes.data)
            else:
                ps.append(None)
        VP = ctypes.c_void_p * self.count
        phi_a = VP(*phis)
        u_a = VP(*us) if any(v is not None for v in us) else None
        p_a = VP(*ps) if any(v is not None for v in ps) else None
        out = ctypes.c_void_p()
        L.check(self.lib.pfl_batch_init(arr, self.count, phi_a, u_a, p_a, ctypes.c_void_p(self.workspace.data_ptr()),
                                        nbytes, ctypes.c_void_p(self.stream.cuda_stream), 1 if tune else 0,
                                        ctypes.byref(out)))
        self.b = out

    def close(self):
        if getattr(self, "b", None):
            self.lib.pfl_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def time(self):
        return self.lib.pfl_batch_time(self.b)

    def step(self, n=1):
        L.check(self.lib.pfl_batch_step(self.b, int(n)))

    def fields(self, i):
        q = self.params[i]
        shape = (q.nz, q.ny, q.nx)
        phi, rho, pr = np.empty(shape), np.empty(shape), np.empty(shape)
        u = np.empty((3,) + shape)
        L.check(self.lib.pfl_batch_fields(self.b, int(i), _ptr(phi), _ptr(rho), _ptr(pr), _ptr(u)))
        return phi, rho, pr, u

    def diag(self, check=True):
        out = np.empty((self.count, 8))
        nf = np.zeros(self.count, dtype=np.int64)
        st = self.lib.pfl_batch_diag(self.b, _ptr(out), _ptr(nf))
        if check:
            L.check(st)
        return out, nf, st

    def shapes(self):
        t = np.zeros(2, dtype=np.int32)
        g = np.zeros(2, dtype=np.int32)
        n = np.zeros(2, dtype=np.int32)
        L.check(self.lib.pfl_batch_shapes(self.b, _ptr(t), _ptr(g), _ptr(n)))
        return t, g, n

    def set_shape(self, cls, tile_x, tile_y, z_chunk=0, grid=0):
        """Launch shape of class cls (0: one z plane, 1: 3-D): tile_x x tile_y
        tiles, z_chunk planes per tile (0: whole lattice), grid blocks (0: SMs x
        resident blocks)."""
        L.check(self.lib.pfl_batch_set_shape(self.b, int(cls), int(tile_x), int(tile_y), int(z_chunk), int(grid)))
