"""Surrogate network, posterior sampler and ESS (include/mjp_surrogate.h).

Argument marshalling only: every step runs in libmjp.so's kernels.  Host
arrays (NumPy) give synchronous calls; the sampler keeps its state on the
device between calls.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import capi
from .capi import MLP_NNORM, MLP_NPAR, PTR_HOST

__all__ = ["MLP", "Sampler", "ess", "MLP_NPAR", "MLP_NNORM", "SI_ADAPT"]

# Adaptive-protocol constants of SI A.4.3.
SI_ADAPT = dict(every=300, window=100, cycle=100, good_cycles=10, z0=1e-8, eps=1e-12, acc_lo=0.2, acc_hi=0.5,
                restart_at_best=1, max_iters=20000)


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data)


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a if shape is None else a.reshape(shape)


class _DeviceView:
    """A float64 device buffer owned by the library, seen through the CUDA
    array interface (no copy)."""

    def __init__(self, ptr: int, shape):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": "<f8", "data": (int(ptr), False),
                                         "version": 3, "strides": None}


class MLP:
    """4 -> 128 -> 128 -> 1 tanh perceptron on the current CUDA device."""

    def __init__(self, seed: int = 0):
        self._h = ctypes.c_void_p()
        capi.check(capi.lib().mjp_mlp_create(ctypes.byref(self._h), ctypes.c_uint64(seed & (2**64 - 1))))

    def set_params(self, params=None, norm=None, stream=None):
        p = None if params is None else np.ascontiguousarray(params, dtype=np.float32)
        n = None if norm is None else _f64(norm)
        if p is not None and p.size != MLP_NPAR or n is not None and n.size != MLP_NNORM:
            raise ValueError("params must hold 17281 values and norm 10")
        capi.check(capi.lib().mjp_mlp_set_params(self._h, None if p is None else _ptr(p),
                                                 None if n is None else _ptr(n), PTR_HOST, _stream(stream)))

    def get_params(self, stream=None):
        p = np.zeros(MLP_NPAR, np.float32)
        n = np.zeros(MLP_NNORM)
        capi.check(capi.lib().mjp_mlp_get_params(self._h, _ptr(p), _ptr(n), PTR_HOST, _stream(stream)))
        return p, n

    def fit_norm(self, psi, y, stream=None):
        ps, yy = _f64(psi, (-1, 4)), _f64(y)
        capi.check(capi.lib().mjp_mlp_fit_norm(self._h, _ptr(ps), _ptr(yy), len(yy), PTR_HOST, _stream(stream)))

    def forward(self, psi, stream=None):
        ps = _f64(psi, (-1, 4))
        out = np.zeros(len(ps))
        capi.check(capi.lib().mjp_mlp_forward(self._h, _ptr(ps), len(ps), _ptr(out), PTR_HOST, _stream(stream)))
        return out

    def loss_grad(self, psi, y, stream=None):
        ps, yy = _f64(psi, (-1, 4)), _f64(y)
        loss = np.zeros(1)
        g = np.zeros(MLP_NPAR, np.float32)
        capi.check(capi.lib().mjp_mlp_loss_grad(self._h, _ptr(ps), _ptr(yy), len(yy), _ptr(loss), _ptr(g), PTR_HOST,
                                                _stream(stream)))
        return float(loss[0]), g

    def train(self, psi, y, steps: int, batch: int, lr: float = 1e-3, beta1: float = 0.9, beta2: float = 0.999,
              eps: float = 1e-8, seed: int = 0, fit_norm: bool = True, stream=None, device_data=False):
        """Adam steps; returns the per-step minibatch losses.  With
        device_data=True, psi and y are CUDA float64 tensors."""
        cfg = capi.TrainCfg(int(steps), int(batch), float(lr), float(beta1), float(beta2), float(eps),
                            ctypes.c_uint64(seed & (2**64 - 1)).value, int(bool(fit_norm)))
        losses = np.zeros(int(steps))
        if device_data:
            import torch
            lt = torch.empty(int(steps), dtype=torch.float64, device=psi.device)
            capi.check(capi.lib().mjp_mlp_train(self._h, ctypes.c_void_p(psi.data_ptr()),
                                                ctypes.c_void_p(y.data_ptr()), int(y.numel()), ctypes.byref(cfg),
                                                ctypes.c_void_p(lt.data_ptr()), capi.PTR_DEVICE, _stream(stream)))
            return lt.cpu().numpy()
        ps, yy = _f64(psi, (-1, 4)), _f64(y)
        capi.check(capi.lib().mjp_mlp_train(self._h, _ptr(ps), _ptr(yy), len(yy), ctypes.byref(cfg), _ptr(losses),
                                            PTR_HOST, _stream(stream)))
        return losses

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            capi.lib().mjp_mlp_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Sampler:
    """MH / delayed-acceptance chains on a 4-rate stencil model and its observations."""

    def __init__(self, model, obs, chains: int, capacity: int, eval_capacity: int = 0, seed: int = 0):
        self._h = ctypes.c_void_p()
        self.model, self.obs = model, obs  # keep them alive
        capi.check(capi.lib().mjp_sampler_create(ctypes.byref(self._h), model._h, obs._h, int(chains),
                                                 int(capacity), int(eval_capacity),
                                                 ctypes.c_uint64(seed & (2**64 - 1))))
        self.chains = int(chains)

    def set_state(self, psi, stream=None):
        ps = _f64(psi, (self.chains, 4))
        capi.check(capi.lib().mjp_sampler_set_state(self._h, _ptr(ps), PTR_HOST, _stream(stream)))

    def get_state(self, stream=None):
        ps = np.zeros((self.chains, 4))
        ll = np.zeros(self.chains)
        capi.check(capi.lib().mjp_sampler_get_state(self._h, _ptr(ps), _ptr(ll), PTR_HOST, _stream(stream)))
        return ps, ll

    def set_cov(self, Z, stream=None):
        z = _f64(Z, (16,))
        capi.check(capi.lib().mjp_sampler_set_cov(self._h, z.ctypes.data_as(capi._f64p), _stream(stream)))

    def get_cov(self, stream=None):
        z = np.zeros(16)
        capi.check(capi.lib().mjp_sampler_get_cov(self._h, z.ctypes.data_as(capi._f64p), _stream(stream)))
        return z.reshape(4, 4)

    def adapt_cov(self, window: int, eps: float = 1e-12, stream=None):
        capi.check(capi.lib().mjp_sampler_adapt_cov(self._h, int(window), float(eps), _stream(stream)))

    def run_plain(self, iters: int, record: bool = True, stream=None):
        capi.check(capi.lib().mjp_sampler_run_plain(self._h, int(iters), int(record), _stream(stream)))

    def run_da(self, net: MLP, iters: int, max_inner: int = 32, record: bool = True, stream=None):
        capi.check(capi.lib().mjp_sampler_run_da(self._h, net._h, int(iters), int(max_inner), int(record),
                                                 _stream(stream)))

    def clear(self, evals: bool = False, stream=None):
        capi.check(capi.lib().mjp_sampler_clear(self._h, int(evals), _stream(stream)))

    def stats(self, stream=None) -> dict:
        st = capi.SamplerStats()
        capi.check(capi.lib().mjp_sampler_stats_get(self._h, ctypes.byref(st), _stream(stream)))
        return {n: int(getattr(st, n)) for n, _ in st._fields_}

    def trace(self, stream=None):
        k = self.stats(stream)["kept"]
        out = np.zeros((self.chains, k, 4))
        if k:
            capi.check(capi.lib().mjp_sampler_trace(self._h, _ptr(out), PTR_HOST, _stream(stream)))
        return out

    def evals(self, stream=None):
        """Kept (psi [n, 4], loglik [n]) pairs as CUDA float64 tensors (copies)."""
        import torch
        p, l = ctypes.c_void_p(), ctypes.c_void_p()
        n = ctypes.c_int64()
        capi.check(capi.lib().mjp_sampler_evals(self._h, ctypes.byref(p), ctypes.byref(l), ctypes.byref(n)))
        m = int(n.value)
        if m == 0:
            return (torch.empty((0, 4), dtype=torch.float64, device="cuda"),
                    torch.empty(0, dtype=torch.float64, device="cuda"))
        torch.cuda.current_stream().synchronize()
        psi = torch.as_tensor(_DeviceView(p.value, (m, 4)), device="cuda").clone()
        ll = torch.as_tensor(_DeviceView(l.value, (m,)), device="cuda").clone()
        return psi, ll

    def checkpoint(self, path=None, net: MLP | None = None, stream=None) -> dict:
        """The sampler's state between runs (mjp_sampler_save: chains, Philox
        counters, counters, kept samples and evaluations, Z) as a byte array,
        with the surrogate's parameters when `net` is given; written to `path`
        (.npz) when one is given, and returned as a dict of arrays."""
        n = ctypes.c_size_t()
        capi.check(capi.lib().mjp_sampler_checkpoint_size(self._h, ctypes.byref(n)))
        blob = np.zeros(int(n.value), dtype=np.uint8)
        capi.check(capi.lib().mjp_sampler_save(self._h, _ptr(blob), blob.nbytes, _stream(stream)))
        d = {"sampler": blob}
        if net is not None:
            d["mlp_params"], d["mlp_norm"] = net.get_params(stream)
        if path is not None:
            np.savez(path, **d)
        return d

    def resume(self, source, net: MLP | None = None, stream=None):
        """Restore a checkpoint (a path written by checkpoint(), or its dict)
        into this sampler, created with the same chains, capacities and seed
        on the same model and observations; and the surrogate's parameters
        into `net` when it is given and the checkpoint holds them."""
        d = source if isinstance(source, dict) else np.load(source)
        blob = np.ascontiguousarray(d["sampler"], dtype=np.uint8)
        capi.check(capi.lib().mjp_sampler_load(self._h, _ptr(blob), blob.nbytes, _stream(stream)))
        if net is not None and "mlp_params" in d:
            net.set_params(d["mlp_params"], d["mlp_norm"], stream)

    def adapt(self, stream=None, **kw) -> dict:
        c = dict(SI_ADAPT)
        c.update(kw)
        cfg = capi.AdaptCfg(int(c["every"]), int(c["window"]), int(c["cycle"]), int(c["good_cycles"]),
                            float(c["z0"]), float(c["eps"]), float(c["acc_lo"]), float(c["acc_hi"]),
                            int(c["restart_at_best"]), int(c["max_iters"]))
        rep = capi.AdaptReport()
        capi.check(capi.lib().mjp_sampler_adapt(self._h, ctypes.byref(cfg), ctypes.byref(rep), _stream(stream)))
        return {"iters": list(rep.iters), "good": list(rep.good), "converged": bool(rep.converged),
                "acc_last": rep.acc_last}

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            capi.lib().mjp_sampler_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ess(trace, stream=None) -> dict:
    """Per-parameter ESS (summed over chains), pooled mean/variance and their
    MCSEs of a trace [chains][len][params] (host array)."""
    tr = _f64(trace)
    C, S, P = tr.shape
    outs = [np.zeros(P) for _ in range(5)]
    capi.check(capi.lib().mjp_ess(_ptr(tr), C, S, P, *[_ptr(o) for o in outs], PTR_HOST, _stream(stream)))
    return dict(zip(("ess", "mean", "var", "mcse_mean", "mcse_var"), outs))


def promoter_initial_psi(obs_groups, chains: int):
    """SI A.4.2 start for the two-state promoter: beta0 = the largest observed
    count, gamma0 = lambda_act0 = lambda_ina0 = 1.5, as Psi = log(theta) for
    every chain.  obs_groups: list over times of (members_list, counts)."""
    top = 0
    for members, counts in obs_groups:
        for mem, c in zip(members, counts):
            if c > 0:
                top = max(top, int(np.min(np.atleast_1d(mem))))
    theta0 = np.array([max(top, 1), 1.5, 1.5, 1.5], dtype=np.float64)
    return np.tile(np.log(theta0), (chains, 1))


def da_vs_plain(model, obs, psi0, chains: int, iters: int, adapt: dict | None = None, train_pairs: int = 65536,
                train_steps: int = 3000, batch: int = 1024, lr: float = 2e-3, max_inner: int = 32, seed: int = 0,
                net_seed: int = 1):
    """The surrogate workflow on one model and data set:

    1. adaptive MH (SI A.2 / A.4.3 constants unless `adapt` overrides them),
       keeping every exact evaluation (Psi', l(Psi'));
    2. train the network on the newest finite pairs (device data, Adam);
    3. from the adapted state with Z frozen, `iters` plain MH iterations and
       `iters` delayed-acceptance iterations, each timed with CUDA events;
    4. ESS, moments and MCSE of both traces (device kernels).

    Returns a dict of timings, counters and statistics."""
    import torch
    cap = max(int(iters), int((adapt or {}).get("window", SI_ADAPT["window"])))
    s = Sampler(model, obs, chains, capacity=cap, eval_capacity=4 * train_pairs + chains * 4000, seed=seed)
    s.set_state(psi0)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)

    def timed(fn):
        torch.cuda.synchronize()
        t0.record()
        fn()
        t1.record()
        torch.cuda.synchronize()
        return t0.elapsed_time(t1) / 1e3

    res = {}
    res["adapt_s"] = timed(lambda: res.__setitem__("adapt", s.adapt(**(adapt or {}))))
    psi_ev, ll_ev = s.evals()
    ok = torch.isfinite(ll_ev)
    psi_ev, ll_ev = psi_ev[ok][-train_pairs:].contiguous(), ll_ev[ok][-train_pairs:].contiguous()
    net = MLP(seed=net_seed)
    res["train_pairs"] = int(ll_ev.numel())
    losses = []
    res["train_s"] = timed(lambda: losses.append(net.train(psi_ev, ll_ev, steps=train_steps, batch=batch, lr=lr,
                                                           seed=seed, fit_norm=True, device_data=True)))
    res["train_loss_first_last"] = [float(losses[0][0]), float(losses[0][-20:].mean())]
    res["Z"] = s.get_cov().tolist()
    psi_a, _ = s.get_state()

    out = {}
    for mode in ("plain", "da"):
        s.set_state(psi_a)
        s.clear()
        if mode == "plain":
            sec = timed(lambda: s.run_plain(iters))
        else:
            sec = timed(lambda: s.run_da(net, iters, max_inner=max_inner))
        tr = s.trace()
        st = s.stats()
        e = ess(tr)
        out[mode] = {"seconds": sec, "stats": st, "trace": tr, **e,
                     "min_ess": float(e["ess"].min()), "ess_per_s": float(e["ess"].min() / sec)}
    res["plain"], res["da"] = out["plain"], out["da"]
    p, d = out["plain"], out["da"]
    res["z_mean"] = (np.abs(d["mean"] - p["mean"]) / np.sqrt(d["mcse_mean"] ** 2 + p["mcse_mean"] ** 2)).tolist()
    res["z_var"] = (np.abs(d["var"] - p["var"]) / np.sqrt(d["mcse_var"] ** 2 + p["mcse_var"] ** 2)).tolist()
    res["ess_per_s_ratio"] = d["ess_per_s"] / p["ess_per_s"]
    return res
