"""GPU parity of batched uneven instances (persistent build, float64
composition, CUDA-graph replay, autotuner) against the FP64 oracle."""
import numpy as np
import pytest

import paper_1304_6514_gb300 as nvp
import workloads
from oracle import nievergelt as nv

from gpu_util import need_gpu, rel_max

pytestmark = pytest.mark.gpu


def _small_batch(seed=11, B=12, P=9):
    st = workloads.Stream(seed)
    mu = st.uniform(B, 0.1, 2.0)
    T = st.uniform(B, 0.5, 2.0)
    S = st.integers(B, 1, 6)
    y0 = st.uniform(2 * B, -2.0, 2.0).reshape(B, 2)
    return mu, T, S, y0, P


def _oracle_instance(mu, T, S, y0, P, dt):
    m = nv.steps_per_slice(0.0, T, int(S), dt)
    nodes = nv.uniform_nodes(-3.0, 3.0, P)
    tab = nv.build_table_2d(nv.rhs_vdp(mu), "rk4", 0.0, T, int(S), m, nodes, nodes)   # [j, p, q, c]
    lam, oob = nv.compose_tables_2d(-3.0, 3.0, tab, y0)
    return tab, lam[-1], oob


def _run_batch(torch, mu, T, S, y0, P, dt, prec, graph=False):
    smp = nvp.samples("bilinear2d", P, (-3.0, -3.0), (3.0, 3.0))
    b = nvp.build_batch("vdp", 2, mu, np.zeros_like(T), T, S, smp, nvp.steps("rk4", dt, 0, prec))
    y0_t = torch.tensor(y0, dtype=torch.float64, device="cuda")
    yT = torch.empty_like(y0_t)
    if graph:
        nvp.batch_run(b, y0_t, yT)
    else:
        nvp.batch_compose(b, y0_t, yT)
    oob = nvp.batch_check(b)
    tabs = nvp.batch_tables(b, torch.float64 if prec == "fp64" else torch.float32).cpu().numpy()
    return b, tabs, yT.cpu().numpy(), oob


def _split_tables(tabs, S, P):
    out, off = [], 0
    for s in S:
        n = int(s) * P * P * 2
        out.append(tabs[off:off + n].reshape(int(s), P, P, 2).transpose(0, 2, 1, 3))  # [j, p, q, c]
        off += n
    return out


@pytest.mark.parametrize("prec,tol_tab,tol_y", [("fp64", 1e-11, 1e-11), ("fp32", 1e-5, 1e-4)])
def test_small_batch_elementwise(prec, tol_tab, tol_y):
    """12 instances, S in 1..6, horizons 0.5..2: every table entry and every
    composed state against the oracle, instance by instance."""
    torch = need_gpu()
    mu, T, S, y0, P = _small_batch()
    dt = 1e-2
    b, tabs, yT, oob = _run_batch(torch, mu, T, S, y0, P, dt, prec)
    parts = _split_tables(tabs, S, P)
    ooob = 0
    for i in range(len(mu)):
        otab, oy, o = _oracle_instance(mu[i], T[i], S[i], y0[i], P, dt)
        ooob += o
        assert rel_max(parts[i], otab) <= tol_tab, i
        assert rel_max(yT[i], oy) <= tol_y, i
    assert oob == ooob
    b.destroy()


def test_graph_replay_and_autotune_are_bitwise_stable():
    """The captured graph and every CTA shape the autotuner tries give the
    same bits: a sample's arithmetic does not depend on the launch shape."""
    torch = need_gpu()
    mu, T, S, y0, P = _small_batch(seed=12, B=20, P=32)
    dt = 1e-2
    b, tabs, yT, _ = _run_batch(torch, mu, T, S, y0, P, dt, "fp32")
    y0_t = torch.tensor(y0, dtype=torch.float64, device="cuda")
    y1 = torch.empty_like(y0_t)
    nvp.batch_run(b, y0_t, y1)
    nvp.batch_run(b, y0_t, y1)        # replay of the captured graph
    nvp.batch_check(b)
    assert np.array_equal(y1.cpu().numpy(), yT)
    best = nvp.batch_autotune(b)
    assert best in (128, 256, 512, 1024)
    nvp.batch_rebuild(b)
    y2 = torch.empty_like(y0_t)
    nvp.batch_compose(b, y0_t, y2)
    nvp.batch_check(b)
    assert np.array_equal(y2.cpu().numpy(), yT)
    assert np.array_equal(nvp.batch_tables(b, torch.float32).cpu().numpy(), tabs)
    b.destroy()


def full_batch_check_instances(vb):
    """Instances of the 4096-instance batch checked element by element: the
    three cheapest, the longest horizon, the most slices, the largest damping
    (its limit cycle leaves [-3,3]^2, so lookups extrapolate) and the two
    instances with the most steps per slice."""
    m = np.ceil(vb.T / vb.S / vb.dt - 1e-9)
    pick = list(np.argsort(vb.T)[:3]) + [int(np.argmax(vb.T)), int(np.argmax(vb.S)), int(np.argmax(vb.mu))]
    pick += list(np.argsort(-m)[:2])
    return list(dict.fromkeys(int(i) for i in pick))


def test_full_batch_sampled_instances():
    """4096 Van der Pol instances (mu ~ U[0.1,2], T ~ U[5,20], S ~ U{8..256},
    32 x 32 grid on [-3,3]^2, RK4 dt = 1e-3, float32 tables, float64
    composition): the instances of full_batch_check_instances (cheap and
    hard: longest horizon, most slices, largest damping with out-of-range
    lookups) checked element by element against the oracle, every table entry
    and the composed final state."""
    torch = need_gpu()
    vb = workloads.vdp_batch()
    P = vb.per_dim
    b, tabs, yT, oob = _run_batch(torch, vb.mu, vb.T, vb.S, vb.y0, P, vb.dt, "fp32")
    info = nvp.batch_info(b)
    assert info["total_slices"] == int(np.sum(vb.S))
    parts_off = np.concatenate([[0], np.cumsum(vb.S.astype(np.int64) * P * P * 2)])
    extrapolated = 0
    for i in full_batch_check_instances(vb):
        otab, oy, o = _oracle_instance(vb.mu[i], vb.T[i], vb.S[i], vb.y0[i], P, vb.dt)
        extrapolated += o
        g = tabs[parts_off[i]:parts_off[i + 1]].reshape(int(vb.S[i]), P, P, 2).transpose(0, 2, 1, 3)
        assert rel_max(g, otab) <= 1e-5, i
        assert rel_max(yT[i], oy) <= 1e-4, (i, rel_max(yT[i], oy))
    assert extrapolated > 0                      # the hard path (EXTRAPOLATE) was among them
    assert oob >= extrapolated
    assert np.all(np.isfinite(yT))
    b.destroy()


def test_full_batch_float64_checked_instances():
    """The same 4096 instances with float64 tables (the float64 method on the
    batch): every table entry and the final state of the checked instances
    within the float64 tolerance, and the float32 batch's final states within
    1e-4 of these over all 4096 instances (its table rounding, amplified by
    up to 256 bilinear lookups)."""
    torch = need_gpu()
    vb = workloads.vdp_batch()
    P = vb.per_dim
    b, tabs, yT, oob = _run_batch(torch, vb.mu, vb.T, vb.S, vb.y0, P, vb.dt, "fp64")
    parts_off = np.concatenate([[0], np.cumsum(vb.S.astype(np.int64) * P * P * 2)])
    for i in full_batch_check_instances(vb):
        otab, oy, _ = _oracle_instance(vb.mu[i], vb.T[i], vb.S[i], vb.y0[i], P, vb.dt)
        g = tabs[parts_off[i]:parts_off[i + 1]].reshape(int(vb.S[i]), P, P, 2).transpose(0, 2, 1, 3)
        assert rel_max(g, otab) <= 1e-11, i
        assert rel_max(yT[i], oy) <= 1e-11, (i, rel_max(yT[i], oy))
    b.destroy()
    b32, _, y32, _ = _run_batch(torch, vb.mu, vb.T, vb.S, vb.y0, P, vb.dt, "fp32")
    err = np.linalg.norm(y32 - yT, axis=1) / np.linalg.norm(yT, axis=1)
    assert err.max() <= 1e-4, err.max()
    b32.destroy()
