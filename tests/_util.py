"""Helpers shared by the GPU tests: build matching meshes for the CUDA library
and the oracle, move arrays between numpy and device tensors."""
import numpy as np

import oracle as O
from paper_2505_00384_gb300 import dgx
from paper_2505_00384_gb300 import inputs

GAMMA = 1.4


def torch_cuda():
    import torch
    return torch


def dev(a, dtype=None):
    torch = torch_cuda()
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def host(t):
    torch = torch_cuda()
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


class Case:
    """A mesh built identically for the CUDA library and the oracle."""

    def __init__(self, nx, ny, nz, r, Lx=1000.0, Ly=1000.0, Lz=1000.0, terrain=0, hc=0.0, ac=1000.0, xc=None,
                 yc=None, bc_lateral=0, refine=None):
        torch = torch_cuda()
        self.m = O.make_mesh(nx, ny, nz, r, Lx=Lx, Ly=Ly, Lz=Lz, terrain=terrain, hc=hc, ac=ac, xc=xc, yc=yc,
                             bc_lateral=bc_lateral, refine=refine)
        self.desc = dgx.mesh_desc(nx, ny, nz, r, Lx, Ly, Lz, terrain=terrain, h_c=hc, a_c=ac, x_c=self.m.xc,
                                  y_c=self.m.yc, bc_lateral=bc_lateral, refine=refine)
        self.stream = torch.cuda.current_stream().cuda_stream
        self.ctx = dgx.dgx_create(0, self.stream)
        dgx.dgx_mesh_build(self.ctx, self.desc)
        self.N = dgx.dgx_num_dofs(self.ctx)
        assert self.N == O.ndofs(self.m)

    def close(self):
        if self.ctx is not None:
            torch_cuda().cuda.synchronize()
            dgx.dgx_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def coords(self):
        return O.node_coords(self.m)

    def random_coefficients(self, seed, rel=0.1):
        """rho, p_k: hydrostatic-like profiles with relative noise (seeded)."""
        X = self.coords()
        rho = inputs.perturbed_profile(X[2], 1.2, 7314.0, rel, seed)
        pk = inputs.perturbed_profile(X[2], 1e5, 7314.0, rel, seed + 1)
        return rho, pk

    def set_coefficients(self, rho, pk, a_dt):
        self._rho = dev(rho)
        self._pk = dev(pk)
        dgx.dgx_set_coefficients(self.ctx, self._rho.data_ptr(), self._pk.data_ptr(), a_dt, GAMMA)


def rel_max_err(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)
