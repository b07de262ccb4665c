"""Helpers shared by the GPU tests: run the CUDA path on a gen.Problem through
the C ABI (Python binding) and bring results back to the host."""
import numpy as np
import torch

import paper_1802_04256_gb300 as R


def t(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def faces(p):
    """The face tractions of a gen.Problem as device tensors (lo, hi, axis,
    coef) for Pattern.add_traction."""
    return (t(p.face_lo), t(p.face_hi), t(p.face_axis, torch.int8), t(p.face_coef))


class GpuRun:
    """Pattern + assembly (+ loads) of one problem on the GPU."""

    def __init__(self, p, loads=True):
        self.p = p
        self.pat = R.Pattern.from_problem(p)
        self.E, self.nu = t(p.E), t(p.nu)
        self.body = t(p.body) if np.any(p.body) else None
        self.K, self.f = self.pat.assemble(self.E, self.nu, self.body)
        if loads and p.n_faces:
            self.pat.add_traction(*faces(p), self.f)
        torch.cuda.synchronize()

    def host_csr(self):
        rowptr, cols = self.pat.csr()
        return rowptr.cpu().numpy(), cols.cpu().numpy()

    def host_K(self):
        return self.K.cpu().numpy()

    def solve(self, rtol=1e-10, max_iter=200000, scale=1e8, precond="jacobi"):
        K = self.K.clone()
        f = self.f.clone()
        alpha = self.pat.apply_penalty(K, f, t(self.p.fixed_dofs, torch.int64), t(self.p.fixed_vals), scale)
        u, it, rr = self.pat.solve_pcg(K, f, rtol=rtol, max_iter=max_iter, precond=precond)
        return u, it, rr, alpha, K, f


def bsr_matvec(rowptr, cols, vals, x):
    """Host reference product of a 3x3-block CSR matrix with x (numpy)."""
    n = len(rowptr) - 1
    x = np.asarray(x).reshape(-1, 3)
    rows = np.repeat(np.arange(n), np.diff(rowptr))
    y = np.einsum("tab,tb->ta", vals.reshape(-1, 3, 3), x[cols])
    out = np.zeros((n, 3))
    np.add.at(out, rows, y)
    return out.ravel()
