"""Torch-facing actor cost map over the C ABI of include/camp_costmap.h.

The MLP of Sec. V-A (observation [x_init; x_ref,0] -> 2 x ``hidden`` ReLU ->
sigmoid scaled to [q_lo, q_hi]) producing the per-stage Q_t of the MPC layer.
Every layer runs in libcamp.so's tensor-core kernel; PyTorch supplies device
memory and streams only.
"""
from __future__ import annotations

import torch

from . import camp


class CostMap:
    """Weights (W1, b1, W2, b2, W3, b3; W_l of shape [n_in_l, n_out_l]) and the
    workspace for batches up to B_max."""

    def __init__(self, weights, N: int, B_max: int, q_lo=0.1, q_hi=10.0, device=None):
        self.device = torch.device(device or "cuda")
        self.N = int(N)
        W = [torch.as_tensor(w, dtype=torch.float32, device=self.device).contiguous() for w in weights]
        self.W1, self.b1, self.W2, self.b2, self.W3, self.b3 = W
        self.hidden = self.W1.shape[1]
        self.n_out = self.W3.shape[1]
        if self.W1.shape[0] != 26 or self.n_out != 13 * self.N:
            raise ValueError("W1 must be [26, hidden] and W3 [hidden, N * 13]")
        self.B_max = int(B_max)
        nbytes = camp.mpc_costmap_workspace_bytes(self.B_max, self.hidden, self.n_out)
        self.ws = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self.net = camp.mpc_costmap(n_in=26, hidden=self.hidden, n_out=self.n_out, W1=self.W1.data_ptr(),
                                    b1=self.b1.data_ptr(), W2=self.W2.data_ptr(), b2=self.b2.data_ptr(),
                                    W3=self.W3.data_ptr(), b3=self.b3.data_ptr(), q_lo=q_lo, q_hi=q_hi)

    def _check(self, B):
        if B > self.B_max:
            raise ValueError(f"batch {B} above B_max {self.B_max}")

    def forward(self, x0, x_ref, Q=None):
        """Q [B, N, 13] (written into ``Q`` when given, e.g. a problem's Q buffer)."""
        B = x0.shape[0]
        self._check(B)
        if Q is None:
            Q = torch.empty(B, self.N, 13, dtype=torch.float32, device=self.device)
        st = torch.cuda.current_stream(self.device).cuda_stream
        camp.check(camp.mpc_costmap_forward(self.net, B, self.N, x0.data_ptr(), x_ref.data_ptr(), Q.data_ptr(),
                                            self.ws.data_ptr(), st), "mpc_costmap_forward")
        return Q

    def backward(self, x0, x_ref, dQ, out=None, with_obs=False):
        """(dW1, db1, dW2, db2, dW3, db3) and dL/do (or None) from dL/dQ."""
        B = x0.shape[0]
        self._check(B)
        if out is None:
            out = [torch.empty_like(t) for t in (self.W1, self.b1, self.W2, self.b2, self.W3, self.b3)]
        d_obs = torch.empty(B, 26, dtype=torch.float32, device=self.device) if with_obs else None
        st = torch.cuda.current_stream(self.device).cuda_stream
        camp.check(camp.mpc_costmap_backward(self.net, B, self.N, x0.data_ptr(), x_ref.data_ptr(),
                                             dQ.contiguous().data_ptr(), self.ws.data_ptr(),
                                             *[t.data_ptr() for t in out], 0 if d_obs is None else d_obs.data_ptr(),
                                             st), "mpc_costmap_backward")
        return out, d_obs

    def wait_flag(self):
        """The workspace's device-wait flag (nonzero: a bounded wait gave up)."""
        return int(self.ws[:4].view(torch.int32).item())
