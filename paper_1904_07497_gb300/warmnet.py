"""Learned warm start for RES-PCA (not in the paper).

The solver's leading iterations, in which S stays 0 and no label moves, are
computed in closed form (ramp skip).  From the state they end in, this module
runs K unrolled layers of the Sec. 4 iteration with the labels fixed and a
learned step rho_k and soft threshold tau_k per layer (respca_net_forward),
then hands the result to the plain solver as a warm start (respca_warm) to
finish to tol.  The per-layer values are log multipliers on the plain
schedule (rho_k = rho kappa^k exp(theta_k), tau_k = exp(phi_k) / rho_k),
predicted by a 2-layer tanh MLP (width 64) from statistics of the ramp-end
iterate; the MLP's output bias alone is the learned per-layer scalars.

Training fits the MLP so that the network's output is close to the plain
solver's converged answer (L*, S*) of each training problem:
    loss = (||L_K - L*||^2 + ||S_K - S*||^2) / ||X||^2,
with exact gradients from the library's reverse pass (respca_net_backward,
respca_mlp_backward) and Adam steps (respca_adam_step).  Everything that
touches a matrix runs in the CUDA library; this module marshals arguments and
does the scalar bookkeeping (feature normalisation, the schedule's chain rule
is in the library).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from . import respca as R

NZ = 6   # statistics fed to the MLP


@dataclass
class RampState:
    L: object
    S: object
    Theta: object
    p: object
    rho: float
    iters: int
    lam: float
    z: np.ndarray            # raw statistics (before normalisation)
    x_norm: float
    stats: dict = field(default_factory=dict)


@dataclass
class Sample:
    X: object
    c: int
    ramp: RampState
    L_star: object
    S_star: object
    plain_iters: int
    plain_ms: float


def _empty_cm(d, n, device):
    import torch
    return torch.empty((n, d), device=device, dtype=torch.float32).T


class WarmStart:
    """MLP -> per-layer (rho_k, tau_k) -> K unrolled layers -> plain solver."""

    def __init__(self, layers: int = 8, hidden: int = 64, rho0: float = 1e-4, kappa: float = 1.5,
                 seed: int = 0, device: int | None = None):
        import torch
        self.K, self.H, self.nout = int(layers), int(hidden), 2 * int(layers)
        self.rho0, self.kappa = float(rho0), float(kappa)
        dev = torch.cuda.current_device() if device is None else device
        self.device = torch.device("cuda", dev)
        self.stream = torch.cuda.current_stream(self.device)
        g = torch.Generator().manual_seed(int(seed))
        W1 = torch.randn(self.H, NZ, generator=g) / math.sqrt(NZ)
        b1 = torch.zeros(self.H)
        W2 = torch.randn(self.nout, self.H, generator=g) * 0.01
        b2 = torch.zeros(self.nout)
        self.params = torch.cat([W1.ravel(), b1, W2.ravel(), b2]).to(self.device).contiguous()
        self.grad = torch.zeros_like(self.params)
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.hidden = torch.zeros(self.H, device=self.device)
        self.out = torch.zeros(self.nout, device=self.device)
        self.zdev = torch.zeros(NZ, device=self.device)
        self.z_mean = np.zeros(NZ)
        self.z_std = np.ones(NZ)
        self.t = 0
        self.ramp_solver = R.Solver(rho0=rho0, kappa=kappa, stop_after_ramp=True, device=dev)
        self.plain = R.Solver(rho0=rho0, kappa=kappa, device=dev)
        self.net = R.respca_net_create(dev, self.stream)

    def close(self):
        if getattr(self, "net", None):
            R.respca_net_destroy(self.net)
            self.net = None
        for s in ("ramp_solver", "plain"):
            if getattr(self, s, None) is not None:
                getattr(self, s).close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------ states
    def ramp_state(self, X, c: int, lam: float = 0.0) -> RampState:
        """The closed-form leading iterations and the MLP's statistics of
        their end state: log rho, log lambda, log(||X||_F / sqrt(dn)),
        log of the residual and step norms relative to ||X||, log(c / n)."""
        d, n = X.shape
        L, S, Th = (_empty_cm(d, n, X.device) for _ in range(3))
        import torch
        p = torch.empty(n, device=X.device, dtype=torch.int32)
        warm = R.respca_warm()
        warm.Theta = Th.data_ptr()
        warm.warm = 0
        st = R.respca_solve(self.ramp_solver.h, X, c, L, S, p, lam=lam, tol=1e-6, max_iter=500, warm=warm)
        x_norm = float(st["x_norm"])
        tiny = 1e-30
        z = np.array([math.log(warm.rho), math.log(st["lambda"]), math.log(x_norm / math.sqrt(d * n) + tiny),
                      math.log(st["err_resid"] + tiny), math.log(st["err_dL"] + tiny), math.log(c / n)])
        return RampState(L, S, Th, p, float(warm.rho), int(st["iters"]), float(st["lambda"]), z, x_norm, st)

    def sample(self, X, c: int, lam: float = 0.0, tol: float = 1e-6) -> Sample:
        """A training example: the ramp-end state and the plain answer."""
        res = self.plain.solve(X, c, lam=lam, tol=tol)
        rs = self.ramp_state(X, c, lam)
        return Sample(X, c, rs, res.L, res.S, int(res.stats["iters"]), float(res.stats["ms_total"]))

    # ------------------------------------------------------------ network
    def multipliers(self, z: np.ndarray) -> list[float]:
        import torch
        zn = (np.asarray(z) - self.z_mean) / self.z_std
        self.zdev.copy_(torch.from_numpy(zn.astype(np.float32)))
        R.respca_mlp_forward(self.params, NZ, self.H, self.nout, self.zdev, self.out, self.hidden,
                             stream=self.stream)
        return self.out.cpu().tolist()

    def schedule(self, rs: RampState, m) -> tuple[list[float], list[float]]:
        return R.respca_net_schedule(rs.rho, self.kappa, m)

    def forward(self, X, c: int, rs: RampState, m, L=None, S=None, Theta=None):
        rho_k, tau_k = self.schedule(rs, m)
        R.respca_net_forward(self.net, X, rs.p, c, rs.lam, rs.S, rs.Theta, rho_k, tau_k, L, S, Theta)
        return rho_k, tau_k

    def fit(self, samples: list[Sample], steps: int = 100, lr: float = 1e-2, log=None) -> list[float]:
        """Adam on the mean loss over `samples`; returns the loss per step."""
        import torch
        Z = np.stack([s.ramp.z for s in samples])
        self.z_mean = Z.mean(axis=0)
        sd = Z.std(axis=0)
        self.z_std = np.where(sd > 1e-6, sd, 1.0)
        gout = torch.zeros(self.nout, device=self.device)
        history = []
        B = len(samples)
        for step in range(steps):
            total = 0.0
            for i, s in enumerate(samples):
                m = self.multipliers(s.ramp.z)
                self.forward(s.X, s.c, s.ramp, m)
                loss, _, _, gm = R.respca_net_backward(self.net, s.L_star, s.S_star,
                                                       1.0 / (B * s.ramp.x_norm ** 2), self.K)
                total += loss
                gout.copy_(torch.tensor(gm, dtype=torch.float32))
                R.respca_mlp_backward(self.params, NZ, self.H, self.nout, self.zdev, self.hidden, gout,
                                      self.grad, accumulate=(i > 0), stream=self.stream)
            self.t += 1
            R.respca_adam_step(self.params, self.grad, self.m, self.v, lr=lr, t=self.t, stream=self.stream)
            history.append(total)
            if log is not None:
                log(step, total)
        return history

    # ------------------------------------------------------------ inference
    def solve(self, X, c: int, lam: float = 0.0, tol: float = 1e-6, max_iter: int = 500, use_net: bool = True,
              storage: int = 0):
        """Ramp (closed form) -> K layers -> plain iterations to tol.
        X may be FP32, BF16 or FP16 (read as given by every phase).  storage 1
        keeps the intermediate layers' S and Theta in BF16 (respca_net_infer);
        the continuation always runs with FP32 state.  Returns (L, S, p, info)
        with the iteration counts of each phase and the wall time of the whole
        call on the stream."""
        import torch
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(self.stream)
        rs = self.ramp_state(X, c, lam)
        d, n = X.shape
        if use_net:
            L, S, Th = (_empty_cm(d, n, X.device) for _ in range(3))
            m = self.multipliers(rs.z)
            rho_k, tau_k = self.schedule(rs, m)
            R.respca_net_infer(self.net, X, rs.p, c, rs.lam, rs.S, rs.Theta, rho_k, tau_k, L, S, Th,
                               storage=storage)
            rho_next, layers = rho_k[-1] * self.kappa, self.K
        else:
            L, S, Th, rho_next, layers = rs.L, rs.S, rs.Theta, rs.rho, 0
        warm = R.respca_warm()
        warm.Theta = Th.data_ptr()
        warm.rho = rho_next
        warm.warm = 1
        p = rs.p
        st = R.respca_solve(self.plain.h, X, c, L, S, p, lam=lam, tol=tol,
                            max_iter=max(0, max_iter - rs.iters - layers), warm=warm)
        ev1.record(self.stream)
        ev1.synchronize()
        # kernels: the two solver calls count their own; with the network the MLP (1),
        # the label sort, the first D sums and 2 per layer
        launches = int(rs.stats["kernel_launches"]) + int(st["kernel_launches"])
        if use_net:
            launches += 1 + 2 + 2 * self.K
        info = dict(ramp_iters=rs.iters, layers=layers, cont_iters=int(st["iters"]), launches=launches,
                    total_iters=rs.iters + layers + int(st["iters"]), converged=int(st["converged"]),
                    err=float(st["err"]), ms=float(ev0.elapsed_time(ev1)))
        return L, S, p, info
