"""Python front end of libmrcm.so: one object per handle.

Device memory for inputs/outputs and the CUDA stream come from PyTorch;
every step of the method runs in the library's CUDA kernels.
"""
from __future__ import annotations

import numpy as np

from . import _lib as L


def _stream_ptr(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


class MRCM:
    """MRCM-OS solver for one problem or an ensemble of problems.

    problems: one object (or a list) with attributes dim, n, h, K, f,
    bc_kind, bc_value (see ``inputs.Problem``); partitions: matching
    (sub, overlap) objects; params: space, alpha_basis, alpha_smooth.
    precision: "fp64" or "mixed".  particular: "omega" (Step 4 on Omega_i,
    the paper's method) or "hat" (the variant on hat-Omega_i with the basis
    factor).  K / f may be numpy arrays (copied from the host) or CUDA
    tensors (copied on the device)."""

    def __init__(self, problems, partitions, space=1, alpha_basis=1.0, alpha_smooth=1.0,
                 precision="fp64", ir_tol=1e-12, max_ir=30, stream=None, device_inputs=False,
                 particular="omega"):
        import torch
        single = not isinstance(problems, (list, tuple))
        self.problems = [problems] if single else list(problems)
        parts = [partitions] * len(self.problems) if not isinstance(partitions, (list, tuple)) \
            else list(partitions)
        self.dim = self.problems[0].dim
        prec = L.MRCM_FP64 if precision == "fp64" else L.MRCM_MIXED
        if particular not in ("omega", "hat"):
            raise ValueError("particular must be 'omega' or 'hat'")
        self.params = L.make_params(space, alpha_basis, alpha_smooth, prec, ir_tol, max_ir,
                                    L.MRCM_PARTICULAR_HAT if particular == "hat" else L.MRCM_PARTICULAR_OMEGA)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        grids, bcs, pts, Ks, fs = [], [], [], [], []
        self._keep = []
        for pr, pt in zip(self.problems, parts):
            g, b, p = L.make_structs(pr.dim, pr.n, pr.h, pr.bc_kind, pr.bc_value, pt.sub, pt.overlap)
            grids.append(g)
            bcs.append(b)
            pts.append(p)
            if device_inputs:
                Kt = torch.as_tensor(np.ascontiguousarray(pr.K, dtype=np.float64)).cuda()
                ft = torch.as_tensor(np.ascontiguousarray(pr.f, dtype=np.float64)).cuda()
                self._keep += [Kt, ft]
                Ks.append(Kt.data_ptr())
                fs.append(ft.data_ptr())
            else:
                Kh = np.ascontiguousarray(pr.K, dtype=np.float64)
                fh = np.ascontiguousarray(pr.f, dtype=np.float64)
                self._keep += [Kh, fh]
                Ks.append(Kh.ctypes.data)
                fs.append(fh.ctypes.data)
        sp = _stream_ptr(self.stream)
        if len(self.problems) == 1:
            self.h = L.mrcm_create(grids[0], Ks[0], fs[0], bcs[0], pts[0], self.params,
                                   int(device_inputs), sp)
        else:
            self.h = L.mrcm_create_batch(grids, Ks, fs, bcs, pts, self.params, int(device_inputs), sp)
        self._keep = []

    def build_basis(self):
        L.mrcm_build_basis(self.h)
        self._version = getattr(self, "_version", 0) + 1

    def solve_interface(self):
        L.mrcm_solve_interface(self.h)
        self._version = getattr(self, "_version", 0) + 1

    def smooth(self, n_steps):
        L.mrcm_smooth(self.h, n_steps)
        self._version = getattr(self, "_version", 0) + 1

    def fluxes(self, member=0, device=False):
        """(p [ncells], u [ncells, 2d]) of one member, x-fastest cell order."""
        pr = self.problems[member]
        nc = int(np.prod(pr.n))
        if device:
            import torch
            p = torch.empty(nc, dtype=torch.float64, device="cuda")
            u = torch.empty((nc, 2 * pr.dim), dtype=torch.float64, device="cuda")
        else:
            p = np.empty(nc)
            u = np.empty((nc, 2 * pr.dim))
        L.mrcm_fluxes(self.h, member, u, p)
        return p, u

    @property
    def ncells(self):
        return int(sum(int(np.prod(pr.n)) for pr in self.problems))

    def state(self):
        """(p [total cells], u [total cells, 2d]) of all members, concatenated
        in member order, as new CUDA tensors."""
        import torch
        nc = self.ncells
        p = torch.empty(nc, dtype=torch.float64, device="cuda")
        u = torch.empty((nc, 2 * self.dim), dtype=torch.float64, device="cuda")
        off = 0
        for m, pr in enumerate(self.problems):
            k = int(np.prod(pr.n))
            L.mrcm_fluxes(self.h, m, u[off:off + k], p[off:off + k])
            off += k
        return p, u

    def set_permeability(self, values, log=False):
        """New K (or log K with log=True) for every cell of every member,
        concatenated in member order; numpy (host) or a CUDA tensor."""
        if not hasattr(values, "data_ptr"):
            values = np.ascontiguousarray(values, dtype=np.float64).reshape(-1)
        L.mrcm_set_permeability(self.h, values, int(log))
        self._version = getattr(self, "_version", 0) + 1

    def adjoint(self, gp=None, gu=None):
        """dL/dlog K [total cells] of a scalar L of the current solution, from
        dL/dp [total cells] and dL/du [total cells, 2d] (either may be None).
        CUDA tensors in, CUDA tensor out; numpy in, numpy out."""
        dev = any(hasattr(a, "data_ptr") for a in (gp, gu) if a is not None)
        if dev or (gp is None and gu is None):
            import torch
            out = torch.empty(self.ncells, dtype=torch.float64, device="cuda")
            gp = gp.contiguous() if gp is not None else None
            gu = gu.contiguous() if gu is not None else None
        else:
            out = np.empty(self.ncells)
            gp = np.ascontiguousarray(gp, dtype=np.float64) if gp is not None else None
            gu = np.ascontiguousarray(gu, dtype=np.float64) if gu is not None else None
        L.mrcm_adjoint(self.h, gp, gu, out)
        return out

    def stats(self):
        return L.mrcm_stats(self.h)

    def profile(self, enable=True):
        L.mrcm_profile(self.h, enable)

    def timings(self):
        return L.mrcm_timings(self.h)

    def close(self):
        if getattr(self, "h", None) is not None:
            L.mrcm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def run(self, n_smooth, graph=False):
        """One full step (basis, interface, n_smooth smoothing steps); graph=True
        replays it as one captured CUDA graph after the first (eager) call."""
        L.mrcm_run(self.h, n_smooth, int(graph))
        self._version = getattr(self, "_version", 0) + 1


def _autograd_function():
    import torch

    class MRCMSolve(torch.autograd.Function):
        """(p, u) = MRCM-OS(log K) with the library's adjoint as backward.

        forward: sets log K, runs one whole step with n_smooth smoothing
        steps and returns the state of all members (concatenated).  backward:
        one mrcm_adjoint call, which reuses the handle's kept factors.  The
        backward must run before the handle solves again."""

        @staticmethod
        def forward(ctx, logK, solver, n_smooth):
            solver.set_permeability(logK.detach().contiguous(), log=True)
            solver.run(n_smooth)
            ctx.solver = solver
            ctx.version = solver._version
            return solver.state()

        @staticmethod
        def backward(ctx, gp, gu):
            solver = ctx.solver
            if solver._version != ctx.version:
                raise RuntimeError("the MRCM handle solved again after this forward; "
                                   "run backward before the next forward on the same handle")
            return solver.adjoint(gp, gu), None, None

    return MRCMSolve


_FN = None


def mrcm_solve(solver, logK, n_smooth):
    """Differentiable MRCM-OS: returns (p, u) of all members for the CUDA
    tensor logK [total cells]; gradients with respect to logK come from the
    hand-written adjoint (mrcm_adjoint)."""
    global _FN
    if _FN is None:
        _FN = _autograd_function()
    return _FN.apply(logK, solver, n_smooth)
