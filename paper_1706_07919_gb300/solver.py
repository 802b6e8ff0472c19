"""Convenience wrapper: one bie_ctx plus torch-allocated device outputs.

Each method calls exactly one entry point of the C ABI (same argument meaning as include/bie.h).
"""
from __future__ import annotations

import numpy as np
import torch

from . import binding as B


class Solver:
    def __init__(self, device: int = 0, stream: torch.cuda.Stream | None = None):
        self.device = device
        self.stream = stream if stream is not None else torch.cuda.current_stream(device)
        self.ctx = B.bie_create(device, self.stream.cuda_stream)
        self.N = 0

    def close(self):
        if self.ctx:
            B.bie_destroy(self.ctx)
            self.ctx = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _dev(self):
        return torch.device("cuda", self.device)

    def set_quadrature(self, ng: int = 4, ng_near: int = 6):
        B.bie_set_quadrature(self.ctx, ng, ng_near)

    def set_geometry(self, nodes, elems, normals, bc):
        B.bie_set_geometry(self.ctx, nodes, elems, normals, bc)
        self.N = int(np.asarray(nodes).shape[0])

    def set_geometry_linear(self, nodes, elems, normals, bc):
        """Linear 3-node elements (elems [E][3]); outputs are per vertex."""
        B.bie_set_geometry_linear(self.ctx, nodes, elems, normals, bc)
        self.N = int(np.asarray(nodes).shape[0])

    def set_option(self, name: str, value: float):
        B.bie_set_option(self.ctx, name, value)

    def set_incident_plane_wave(self, direction):
        B.bie_set_incident_plane_wave(self.ctx, direction)

    def assemble(self, k: float):
        A = torch.empty((self.N, self.N), dtype=torch.complex128, device=self._dev())
        b = torch.empty((self.N,), dtype=torch.complex128, device=self._dev())
        B.bie_assemble(self.ctx, k, A, b)
        return A, b

    def solve_frequencies(self, k, mode: int = B.BIE_MODE_FP64, out=None):
        k = np.ascontiguousarray(k, np.float64)
        surf = out if out is not None else torch.empty((k.shape[0], 2, self.N), dtype=torch.complex128,
                                                       device=self._dev())
        rep = B.bie_solve_frequencies(self.ctx, k, mode, surf)
        return surf, rep

    def solve_frequencies_async(self, k, out=None):
        """Mixed-precision solves enqueued on the context's stream (bie_solve_frequencies_async):
        returns (surf, pending) at once; pending.reports() waits for the stream's work and returns
        the reports.  surf is written in stream order: keep it until then too."""
        k = np.ascontiguousarray(k, np.float64)
        surf = out if out is not None else torch.empty((k.shape[0], 2, self.N), dtype=torch.complex128,
                                                       device=self._dev())
        pending = B.bie_solve_frequencies_async(self.ctx, k, B.BIE_MODE_MIXED, surf, self.stream)
        return surf, pending

    def solve_frequencies_multi(self, k, dirs, mode: int = B.BIE_MODE_MIXED, out=None):
        """Surface solutions [Nk][ndir][2][N] for several incident directions sharing each factor."""
        k = np.ascontiguousarray(k, np.float64)
        nd = np.atleast_2d(dirs).shape[0]
        surf = out if out is not None else torch.empty((k.shape[0], nd, 2, self.N), dtype=torch.complex128,
                                                       device=self._dev())
        rep = B.bie_solve_frequencies_multi(self.ctx, k, dirs, mode, surf)
        return surf, rep

    def eval_field(self, xobs: torch.Tensor, k, surf: torch.Tensor, mode: int = B.BIE_MODE_FP64, out=None):
        k = np.ascontiguousarray(k, np.float64)
        T = out if out is not None else torch.empty((k.shape[0], xobs.shape[0]), dtype=torch.complex128,
                                                    device=self._dev())
        B.bie_eval_field(self.ctx, xobs, k, surf, mode, T)
        return T

    def pulse_spectrum(self, s: torch.Tensor, out=None):
        S = out if out is not None else torch.empty((s.shape[0], s.shape[1] // 2 + 1), dtype=torch.complex128,
                                                    device=self._dev())
        B.bie_pulse_spectrum(self.ctx, s, S)
        return S

    def synthesize(self, T: torch.Tensor, midx, S: torch.Tensor, Nt: int, out_dtype=torch.float64, out=None):
        code = 0 if out_dtype == torch.float64 else 1
        o = out if out is not None else torch.empty((S.shape[0], T.shape[1], Nt), dtype=out_dtype,
                                                    device=self._dev())
        B.bie_synthesize(self.ctx, T, midx, S, Nt, o, code)
        return o

    def top_frequencies(self, S: torch.Tensor, Nt: int, K: int):
        return B.bie_top_frequencies(self.ctx, S, Nt, K)

    # ---- learned warm start (BIE_MODE_LEARNED's network) ----
    def mlp_set_params(self, theta):
        B.bie_mlp_set_params(self.ctx, theta)

    def mlp_get_params(self):
        return B.bie_mlp_get_params(self.ctx)

    def mlp_features(self, k):
        k = np.ascontiguousarray(np.atleast_1d(k), np.float64)
        phi = torch.empty((k.shape[0], self.N, 64), dtype=torch.float32, device=self._dev())
        B.bie_mlp_features(self.ctx, k, phi)
        return phi

    def mlp_forward(self, X: torch.Tensor):
        Y = torch.empty((X.shape[0], 2), dtype=torch.float32, device=self._dev())
        B.bie_mlp_forward(self.ctx, X, Y)
        return Y

    def mlp_loss_grad(self, X: torch.Tensor, T: torch.Tensor):
        g = torch.empty((B.BIE_MLP_PARAMS,), dtype=torch.float32, device=self._dev())
        L = torch.empty((1,), dtype=torch.float32, device=self._dev())
        B.bie_mlp_loss_grad(self.ctx, X, T, g, L)
        return float(L.item()), g

    def mlp_adam_step(self, grad: torch.Tensor, lr: float):
        B.bie_mlp_adam_step(self.ctx, grad, lr)

    def mlp_train(self, k, surf: torch.Tensor, epochs: int):
        return B.bie_mlp_train(self.ctx, k, surf, epochs)

    def mlp_predict(self, k):
        k = np.ascontiguousarray(np.atleast_1d(k), np.float64)
        x0 = torch.empty((k.shape[0], self.N), dtype=torch.complex128, device=self._dev())
        B.bie_mlp_predict(self.ctx, k, x0)
        return x0

    def learned_info(self) -> dict:
        return B.bie_get_learned_info(self.ctx)
