"""Helpers that run the CUDA path through the C-ABI and the FP64 oracle on the same inputs."""
import numpy as np

import oracle

GRAD_MAP = {"deps": "eps", "dq_mean": "dq_mean", "dq_logstd": "dq_logstd", "dW": "dW",
            "dbias": "dbias", "dC": "dC", "dz": "dz"}


def gpu_run(p, precision="fp32", grads=True, grad_out=None, want=None):
    import torch
    from paper_1806_08593_gb300.tmc import Plan
    plan = Plan.from_problem(p, precision)
    t = plan.to_device(p)
    lp = plan.forward(t)
    out = {"log_phat": None}
    if grads:
        go = None if grad_out is None else torch.as_tensor(grad_out, dtype=torch.float64, device="cuda")
        want = want or ("dz", "deps", "dq_mean", "dq_logstd", "dW", "dbias", "dC") + \
            (("dq_A",) if p.q_A is not None else ())
        g = plan.backward(t, grad_out=go, want=want)
        out.update({k: v.cpu().numpy().astype(np.float64) for k, v in g.items()})
    torch.cuda.synchronize()
    plan.sync_status()
    out["log_phat"] = lp.cpu().numpy()
    plan.close()
    return out


def oracle_deps(p, g):
    """d/d eps = exp(logs) * dz, from the oracle's dz (latent by latent: K_i x d_i blocks)."""
    s = np.exp(p.q_logstd.astype(np.float64))
    out = np.empty_like(g["dz"])
    oe = oq = 0
    for K, d in zip(p.K_nodes().astype(int), p.d_nodes().astype(int)):
        out[oe:oe + K * d] = (g["dz"][oe:oe + K * d].reshape(K, d) * s[oq:oq + d]).ravel()
        oe += K * d
        oq += d
    return out


def oracle_run(p, grad_out=None):
    g = oracle.grad(p, grad_out=grad_out)
    g["deps"] = oracle_deps(p, g)
    return g


def rel_err(a, b):
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / nb) if nb > 0 else float(np.linalg.norm(a))


def compare(p, got, ref, tol_logp, tol_grad, keys=None):
    """Element-wise log P check and per-tensor relative-norm gradient check."""
    err = np.abs(got["log_phat"] - ref["log_phat"])
    assert np.all(np.isfinite(got["log_phat"]))
    assert err.max() <= tol_logp, ("log_phat", float(err.max()), int(err.argmax()))
    report = {"log_phat_max_abs": float(err.max())}
    for k in keys or [k for k in got if k != "log_phat"]:
        e = rel_err(got[k], ref[k])
        report[k] = e
        assert np.all(np.isfinite(got[k])), k
        assert e <= tol_grad, (k, e)
    return report


def mixed_roots_problem(seed=31337):
    """One batch whose instances reach the root kernel in different ways: two wide roots (100
    and 70 children, so the plan sums every root's children in chunks), small uneven trees, a
    chain, and a single latent (a root with no children), with a different K and d per
    instance (so the chunk sums' row stride, the largest K, exceeds most roots' K)."""
    from paper_1806_08593_gb300 import workload as wl
    rng = np.random.default_rng(seed)
    parents = [np.array([-1] + [0] * 100, dtype=np.int32), wl.random_tree(rng, 7, 3),
               np.array([-1], dtype=np.int32), wl.chain_parents(3),
               np.array([-1] + [0] * 70, dtype=np.int32), wl.random_tree(rng, 5, 2)]
    Ks = [96, 40, 33, 128, 17, 64]
    ds = [2, 5, 3, 8, 1, 70]
    return wl.make_problem(parents, Ks, ds, [2 * d for d in ds], shared=False, seed=seed)
