"""Reverse-mode differentiation through the entanglement-aware two-site update.

The paper differentiates nothing.  This module makes its update a differentiable function of
the two-site block so that circuit parameters can be optimised through a truncated simulation:

* ``gemm``: complex matrix product (the library's tensor-core contraction) with its backward
  (two more contractions);
* ``tsvd``: the two-site update of the "Entanglement-aware" section as a function of the block
  theta (m x n): full thin SVD by one-sided Jacobi, the cut against a target, and the outputs of
  a rightward update A_q = U_k, A_p = diag(s_k / sqrt(W_k)) V_k^H.  Its backward is the complex
  SVD adjoint with the gauge term and the coupling to the discarded values, in the library's
  kernels (``mps_tsvd_backward_device``);
* ``DiffMPS``: a mixed-canonical MPS driven only by these two functions.  Centre moves are
  updates with no cut; a gate on (q, q+1) moves the centre to q, contracts theta, applies the
  gate and takes the update with the cut (the global schedule of the paper's Fig. 1 for the
  target); ``energy_zz`` sweeps the centre and sums <Z_i Z_{i+1}> from theta at the centre.

Every contraction, SVD and SVD derivative runs in the library's kernels through its C ABI;
PyTorch provides the tensors, views and copies, and chains the derivatives.  Values at or below
``rank_tol`` times the largest are never kept, so every kept value is nonzero and the derivative
exists; for the untruncated simulation the values dropped that way are zero up to rounding.
"""
from __future__ import annotations

import time

import numpy as np
import torch

from . import (FP64, GLOBAL, MPS, TF32X3, mps_gemm_device, mps_schedule_target, mps_tsvd_backward_device,
               mps_tsvd_device)

__all__ = ["Workspace", "gemm", "tsvd", "DiffMPS", "ansatz_gates_torch", "energy_and_grad_ad"]


class Workspace:
    """Scratch and stream for the stateless update calls: a handle sized for chains of
    ``n_qubits`` sites with bonds up to ``chi_max``, on torch's current stream."""

    def __init__(self, n_qubits: int, chi_max: int, precision: int = TF32X3, svd_kernel: int | None = None):
        self.stream = torch.cuda.current_stream()
        self.mps = MPS(max(n_qubits, 2), chi_max=chi_max, precision=precision, log_truncations=False,
                       stream=self.stream.cuda_stream, svd_kernel=svd_kernel)
        self.h = self.mps.h
        self.dtype = torch.complex128 if precision == FP64 else torch.complex64

    def close(self):
        self.mps.close()


def _gemm_raw(ws: Workspace, a: torch.Tensor, b: torch.Tensor, conj_a: bool = False, trans_a: bool = False,
              conj_b: bool = False, trans_b: bool = False) -> torch.Tensor:
    """op(a) op(b) for contiguous 2-D a, b; trans means the transposed operand."""
    ar, ac = a.shape
    br, bc = b.shape
    M, K = (ac, ar) if trans_a else (ar, ac)
    K2, N = (bc, br) if trans_b else (br, bc)
    assert K == K2
    out = torch.empty((M, N), dtype=ws.dtype, device=a.device)
    a_rs, a_cs = (1, ac) if trans_a else (ac, 1)
    b_rs, b_cs = (1, bc) if trans_b else (bc, 1)
    mps_gemm_device(ws.h, M, N, K, a.data_ptr(), a_rs, a_cs, int(conj_a), b.data_ptr(), b_rs, b_cs, int(conj_b),
                    out.data_ptr(), N, 1)
    return out


class _Gemm(torch.autograd.Function):
    @staticmethod
    def forward(ctx, a, b, ws):
        a = a.contiguous()
        b = b.contiguous()
        ctx.ws = ws
        ctx.save_for_backward(a, b)
        return _gemm_raw(ws, a, b)

    @staticmethod
    def backward(ctx, gc):
        a, b = ctx.saved_tensors
        gc = gc.contiguous()
        ga = gb = None
        if ctx.needs_input_grad[0]:
            ga = _gemm_raw(ctx.ws, gc, b, conj_b=True, trans_b=True)      # dC B^H
        if ctx.needs_input_grad[1]:
            gb = _gemm_raw(ctx.ws, a, gc, conj_a=True, trans_a=True)      # A^H dC
        return ga, gb, None


def gemm(ws: Workspace, a: torch.Tensor, b: torch.Tensor) -> torch.Tensor:
    """a @ b (complex, 2-D) in the library's contraction, differentiable."""
    return _Gemm.apply(a.to(ws.dtype), b.to(ws.dtype), ws)


class _TSVD(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, ws, target, max_k, rank_tol, eps, info):
        theta = theta.contiguous()
        m, n = theta.shape
        c = min(m, n)
        dev = theta.device
        u = torch.empty((m, c), dtype=ws.dtype, device=dev)
        s = torch.empty(c, dtype=torch.float64, device=dev)
        v = torch.empty((n, c), dtype=ws.dtype, device=dev)
        aq = torch.empty(m * c, dtype=ws.dtype, device=dev)
        ap = torch.empty(c * n, dtype=ws.dtype, device=dev)
        k, f, w, wk = mps_tsvd_device(ws.h, m, n, theta.data_ptr(), n, target, max_k, rank_tol, u.data_ptr(),
                                      s.data_ptr(), v.data_ptr(), aq.data_ptr(), ap.data_ptr())
        info.update(k=k, f=f, W=w, W_k=wk)
        ctx.ws, ctx.k, ctx.eps, ctx.mn = ws, k, eps, (m, n)
        ctx.save_for_backward(u, s, v)
        return aq[:m * k].view(m, k), ap[:k * n].view(k, n)

    @staticmethod
    def backward(ctx, gq, gp):
        u, s, v = ctx.saved_tensors
        m, n = ctx.mn
        k = ctx.k
        gq = gq.contiguous() if gq is not None else None
        gp = gp.contiguous() if gp is not None else None
        ga = torch.empty((m, n), dtype=ctx.ws.dtype, device=u.device)
        mps_tsvd_backward_device(ctx.ws.h, m, n, k, u.data_ptr(), s.data_ptr(), v.data_ptr(),
                                 gq.data_ptr() if gq is not None else 0, gp.data_ptr() if gp is not None else 0,
                                 ctx.eps, ga.data_ptr())
        return ga, None, None, None, None, None, None


def tsvd(ws: Workspace, theta: torch.Tensor, target: float = 1.0, max_k: int = 0, rank_tol: float = 1e-6,
         eps: float = 0.0):
    """(A_q, A_p, info) of the update of theta (m x n): A_q = U_k (m x k), A_p = diag(s_k/sqrt(W_k)) V_k^H
    (k x n); info = {k, f = W_k/W, W, W_k}.  Differentiable in theta."""
    info = {}
    aq, ap = _TSVD.apply(theta.to(ws.dtype), ws, float(target), int(max_k), float(rank_tol), float(eps), info)
    return aq, ap, info


_ZW = torch.tensor([1.0, -1.0, -1.0, 1.0], dtype=torch.float64)


class DiffMPS:
    """A pure-state MPS whose every step is the differentiable update (see module docstring)."""

    def __init__(self, n_qubits: int, f_min: float = 1.0, n_2q: int = 0, chi_max: int = 256,
                 precision: int = TF32X3, rank_tol: float | None = None, eps: float = 0.0, ws: Workspace = None):
        self.n = n_qubits
        self.ws = ws or Workspace(n_qubits, chi_max, precision)
        self.own_ws = ws is None
        self.chi_max = chi_max
        self.f_min, self.n_2q = f_min, n_2q
        self.rank_tol = (1e-12 if precision == FP64 else 1e-6) if rank_tol is None else rank_tol
        self.eps = eps
        dev = torch.device("cuda", torch.cuda.current_device())
        e0 = torch.zeros((1, 2, 1), dtype=self.ws.dtype, device=dev)
        e0[0, 0, 0] = 1.0
        self.sites = [e0.clone() for _ in range(n_qubits)]
        self.centre = 0
        self.product = 1.0
        self.n_done = 0
        self.k_log = []
        self.records = []
        self.tsvd_calls = 0
        self._replay = None      # iterator over recorded k while a checkpointed layer is recomputed
        self._layer_ks = None    # k of every update of the layer being run for the first time

    def close(self):
        if self.own_ws:
            self.ws.close()

    def _tsvd(self, a2, target):
        self.tsvd_calls += 1
        if self._replay is not None:
            # recomputation of a checkpointed layer: the k of the first run, no new decision
            k = next(self._replay)
            aq, ap, info = tsvd(self.ws, a2, 1.0, k, 0.0, self.eps)
            if info["k"] != k:
                raise RuntimeError("recomputed update kept %d values, the first run %d" % (info["k"], k))
            return aq, ap, info
        aq, ap, info = tsvd(self.ws, a2, target, self.chi_max, self.rank_tol, self.eps)
        self.k_log.append(info["k"])
        if self._layer_ks is not None:
            self._layer_ks.append(info["k"])
        return aq, ap, info

    def target(self) -> float:
        """Global schedule before truncation j+1, evaluated by the library (mps_schedule_target):
        (F_min / P_j)^(1/(n - j)), 1 once P_j < F_min.  P_j is the product of the f values the
        update calls returned, multiplied in gate order in IEEE double precision as the engine's
        device product is."""
        return mps_schedule_target(GLOBAL, self.f_min, self.n_2q, self.n_done, self.product)

    def move_right(self):
        c = self.centre
        a = self.sites[c]
        cl, _, cr = a.shape
        aq, ap, info = self._tsvd(a.reshape(cl * 2, cr), 1.0)
        k = info["k"]
        self.sites[c] = aq.reshape(cl, 2, k)
        b = self.sites[c + 1]
        self.sites[c + 1] = gemm(self.ws, ap, b.reshape(cr, -1)).reshape(k, 2, b.shape[2])
        self.centre = c + 1

    def move_left(self):
        c = self.centre
        a = self.sites[c]
        cl, _, cr = a.shape
        aq, ap, info = self._tsvd(a.reshape(cl, 2 * cr).mH, 1.0)     # M^H = Aq Ap: M = Ap^H Aq^H
        k = info["k"]
        self.sites[c] = aq.mH.reshape(k, 2, cr)
        b = self.sites[c - 1]
        self.sites[c - 1] = gemm(self.ws, b.reshape(-1, cl), ap.mH).reshape(b.shape[0], 2, k)
        self.centre = c - 1

    def move_to(self, q: int):
        while self.centre < q:
            self.move_right()
        while self.centre > q:
            self.move_left()

    def apply_2q(self, q: int, g: torch.Tensor) -> dict:
        """Gate g (4 x 4 tensor, may require grad) on (q, q+1)."""
        self.move_to(q)
        a, b = self.sites[q], self.sites[q + 1]
        cl, cr = a.shape[0], b.shape[2]
        theta = gemm(self.ws, a.reshape(cl * 2, -1), b.reshape(b.shape[0], -1))          # (cl 2) x (2 cr)
        x = theta.reshape(cl, 4, cr).permute(1, 0, 2).reshape(4, cl * cr)
        y = gemm(self.ws, g, x).reshape(4, cl, cr).permute(1, 0, 2).reshape(cl * 2, 2 * cr)
        replay = self._replay is not None
        f_t = 1.0 if replay else self.target()
        aq, ap, info = self._tsvd(y, f_t)
        k = info["k"]
        self.sites[q] = aq.reshape(cl, 2, k)
        self.sites[q + 1] = ap.reshape(k, 2, cr)
        self.centre = q + 1
        rec = dict(info, q=q, f_t=f_t)
        if not replay:
            self.product *= info["f"]
            self.n_done += 1
            self.records.append(rec)
        return rec

    def run_layer(self, gates, checkpoint: bool = False):
        """Apply [(q, g), ...].  With checkpoint, only the layer's input sites are kept for the
        backward; the layer (centre moves, theta, gates, SVDs) is recomputed when the backward
        reaches it, with every k as in the first run."""
        if not checkpoint:
            for q, g in gates:
                self.apply_2q(q, g)
            return
        from torch.utils.checkpoint import checkpoint as _checkpoint
        n = self.n
        qs = [q for q, _ in gates]
        centre0 = self.centre
        ks = []
        first = [True]

        def layer(*tensors):
            live = (self.sites, self.centre)
            replay = not first[0]
            self.sites, self.centre = list(tensors[:n]), centre0
            if replay:
                self._replay = iter(ks)
            else:
                self._layer_ks = ks
            try:
                for q, g in zip(qs, tensors[n:]):
                    self.apply_2q(q, g)
                out = tuple(self.sites)
            finally:
                # a recomputation may also be cut short by the checkpoint machinery (it stops once
                # every tensor it needs exists): the live state comes back in every case
                self._replay = None
                self._layer_ks = None
                if replay:
                    self.sites, self.centre = live
            first[0] = False
            return out

        self.sites = list(_checkpoint(layer, *self.sites, *[g for _, g in gates], use_reentrant=False))

    def energy_zz(self) -> torch.Tensor:
        """sum_i <Z_i Z_{i+1}> (differentiable), the centre sweeping from site 0."""
        self.move_to(0)
        zw = _ZW.to(self.sites[0].device)
        e = None
        for i in range(self.n - 1):
            self.move_to(i)
            a, b = self.sites[i], self.sites[i + 1]
            t = gemm(self.ws, a.reshape(-1, a.shape[2]), b.reshape(b.shape[0], -1)).reshape(a.shape[0], 4, b.shape[2])
            term = ((t.real.double() ** 2 + t.imag.double() ** 2) * zw[None, :, None]).sum()
            e = term if e is None else e + term
        return e

    def bond_dims(self):
        return [int(a.shape[2]) for a in self.sites[:-1]]


def _ry(t):
    c, s = torch.cos(t / 2), torch.sin(t / 2)
    return torch.stack([torch.stack([c, -s]), torch.stack([s, c])]).to(torch.complex128)


def _rz(t):
    z = torch.zeros((), dtype=torch.float64, device=t.device)
    a = torch.exp(torch.complex(z, -0.5 * t))
    b = torch.exp(torch.complex(z, 0.5 * t))
    zero = torch.zeros((), dtype=torch.complex128, device=t.device)
    return torch.stack([torch.stack([a, zero]), torch.stack([zero, b])])


def _rzz(t):
    z = torch.zeros((), dtype=torch.float64, device=t.device)
    a = torch.exp(torch.complex(z, -0.5 * t))
    b = torch.exp(torch.complex(z, 0.5 * t))
    return torch.diag(torch.stack([a, b, b, a]))


def ansatz_gates_torch(n_qubits: int, layers: int, params: torch.Tensor):
    """[(q, 4x4 complex128 gate)] of the layered ansatz (RY, RZ on every qubit, then RZZ on (0,1) ...
    (n-2,n-1), single-qubit rotations folded into the first gate that touches each qubit), as
    differentiable functions of params (layers x (3n - 1): n RY, n RZ, n-1 RZZ angles per layer)."""
    p = params.reshape(layers, 3 * n_qubits - 1)
    eye = torch.eye(2, dtype=torch.complex128, device=params.device)
    out = []
    for l in range(layers):
        ry, rz, zz = p[l, :n_qubits], p[l, n_qubits:2 * n_qubits], p[l, 2 * n_qubits:]
        r = [_rz(rz[i]) @ _ry(ry[i]) for i in range(n_qubits)]
        for i in range(n_qubits - 1):
            local = torch.kron(r[0], r[1]) if i == 0 else torch.kron(eye, r[i + 1])
            out.append((i, _rzz(zz[i]) @ local))
    return out


def energy_and_grad_ad(n_qubits: int, layers: int, params, f_min: float = 1.0, chi_max: int = 256,
                       precision: int = TF32X3, eps: float = 0.0, ws: Workspace = None, checkpoint: bool = False):
    """Energy sum_i <Z_i Z_{i+1}> of the ansatz state and its gradient by reverse mode through the
    truncated simulation (checkpoint: per layer, recomputed in the backward).  Returns (energy,
    grad (numpy, shape of params), info dict)."""
    dev = torch.device("cuda", torch.cuda.current_device())
    p = torch.as_tensor(np.asarray(params, dtype=np.float64), device=dev).clone().requires_grad_(True)
    gates = ansatz_gates_torch(n_qubits, layers, p)
    m = DiffMPS(n_qubits, f_min=f_min, n_2q=len(gates), chi_max=chi_max, precision=precision, eps=eps, ws=ws)
    try:
        t0 = time.perf_counter()
        per = n_qubits - 1
        for l in range(layers):
            m.run_layer(gates[l * per:(l + 1) * per], checkpoint)
        e = m.energy_zz()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        e.backward()
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        info = {"fidelity": m.product, "k_log": list(m.k_log), "bond_dims": m.bond_dims(),
                "max_bond": max(m.bond_dims()), "records": m.records, "forward_s": t1 - t0, "backward_s": t2 - t1,
                "updates": len(m.k_log), "tsvd_calls": m.tsvd_calls}
        return float(e.detach()), p.grad.detach().cpu().numpy().reshape(np.shape(params)), info
    finally:
        m.close()
