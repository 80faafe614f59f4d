"""Chained products C_w <- U_{idx[t,w]} C_w (the step loop of Alg. 1) on the GPU,
checked step by step against the oracle, plus the unitarity-drift measure."""
import numpy as np
import pytest

import oracle
import paper_2203_09353_gb300 as bg
from paper_2203_09353_gb300 import synth

from gpu_util import TOL_FP64, TOL_SPLIT, dev, host

pytestmark = pytest.mark.gpu


def layout(chain):
    """Pool, pool sizes and offsets, states, state offsets, global pool indices."""
    return synth.chain_layout(chain)


def oracle_chain(chain, steps):
    out = []
    for w in range(chain.walkers):
        n = int(chain.n_walker[w])
        C = chain.C0[w].copy()
        for t in range(steps):
            U = chain.pools[n][chain.idx[t, w]]
            C = oracle.matmul(U, C)
        out.append(C)
    return out


def small_chain():
    return synth.annealing_chain(walkers_small=6, walkers_large=2, n_small=32, n_large=96, steps=5,
                         pool_small=4, pool_large=3)


@pytest.mark.parametrize("mode,s", [("fp64", 0), ("split", 9), ("split", 6), ("split", 3)])
@pytest.mark.parametrize("graph", [False, True])
def test_chain_matches_oracle(gpu, mode, s, graph):
    ch = small_chain()
    pool, pn, po, states, wo, gidx = layout(ch)
    prec = bg.precision(mode, s)
    flags = bg.BG_PLAN_CAPTURE_GRAPH if graph else 0
    plan = bg.chain_plan("c128", ch.n_walker, wo, pn, po, prec, flags)
    ping, pong = dev(states), dev(np.zeros_like(states))
    steps = ch.steps
    bg.chain_step(plan, dev(pool), dev(gidx), ping, pong, steps)
    res = host(ping if steps % 2 == 0 else pong)
    ref = oracle_chain(ch, steps)
    tol = TOL_FP64 if mode == "fp64" else TOL_SPLIT[s]
    for w in range(ch.walkers):
        n = int(ch.n_walker[w])
        got = res[wo[w]:wo[w] + n * n].reshape(n, n).T
        # the product of unitaries has ||.||_F = sqrt(n); steps compound the per-step error
        err = np.linalg.norm(got - ref[w]) / n
        assert err <= tol * steps, (w, err)


def test_chain_step_local_parity_and_drift(gpu):
    """Each single step equals oracle(U @ C_gpu_prev); drift ||C^H C - I||_F after the run."""
    import torch
    ch = small_chain()
    pool, pn, po, states, wo, gidx = layout(ch)
    plan = bg.chain_plan("c128", ch.n_walker, wo, pn, po, bg.precision("split", 9))
    cur = states.copy()
    dpool = dev(pool)
    for t in range(ch.steps):
        ping, pong = dev(cur), dev(np.zeros_like(cur))
        bg.chain_step(plan, dpool, dev(gidx[t:t + 1]), ping, pong, 1)
        nxt = host(pong)
        for w in range(ch.walkers):
            n = int(ch.n_walker[w])
            prev = cur[wo[w]:wo[w] + n * n].reshape(n, n).T
            U = ch.pools[n][ch.idx[t, w]]
            ref = oracle.matmul(U, prev)
            got = nxt[wo[w]:wo[w] + n * n].reshape(n, n).T
            assert np.linalg.norm(got - ref) / (np.linalg.norm(U) * np.linalg.norm(prev)) <= 1e-12
        cur = nxt
    dn = torch.tensor(ch.n_walker, dtype=torch.int64, device="cuda")
    do = torch.tensor(wo, dtype=torch.int64, device="cuda")
    out = torch.zeros(ch.walkers, dtype=torch.float64, device="cuda")
    bg.unitarity_drift("c128", dn, do, dev(cur), out, ch.walkers)
    drift = host(out)
    for w in range(ch.walkers):
        n = int(ch.n_walker[w])
        C = cur[wo[w]:wo[w] + n * n].reshape(n, n).T
        assert abs(drift[w] - oracle.unitarity_drift(C)) <= 1e-12 + 1e-6 * drift[w]
        assert drift[w] < 1e-11


def test_chain_real_fp64(gpu):
    rng = np.random.default_rng(5)
    n, W, P, T = 40, 5, 3, 4
    pool = [np.linalg.qr(rng.standard_normal((n, n)))[0] for _ in range(P)]
    C0 = [np.linalg.qr(rng.standard_normal((n, n)))[0] for _ in range(W)]
    idx = rng.integers(0, P, (T, W)).astype(np.int32)
    pf = np.concatenate([np.asfortranarray(U).ravel(order="F") for U in pool])
    sf = np.concatenate([np.asfortranarray(C).ravel(order="F") for C in C0])
    po = np.arange(P) * n * n
    wo = np.arange(W) * n * n
    for mode, s in (("fp64", 0), ("split", 9)):
        plan = bg.chain_plan("r64", [n] * W, wo, [n] * P, po, bg.precision(mode, s))
        ping, pong = dev(sf), dev(np.zeros_like(sf))
        bg.chain_step(plan, dev(pf), dev(idx), ping, pong, T)
        res = host(ping)
        for w in range(W):
            C = C0[w]
            for t in range(T):
                C = oracle.matmul(pool[idx[t, w]], C)
            got = res[wo[w]:wo[w] + n * n].reshape(n, n).T
            assert np.linalg.norm(got - C) / n <= 1e-13
