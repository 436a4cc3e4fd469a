"""GPU tests of the runtime history (klr_argmin_history): answers from the
history equal the evaluated answers bit for bit, kernels whose queries all
hit are not evaluated, misses are evaluated exactly as klr_argmin evaluates
them, and a full table only loses recordings, never correctness."""
import numpy as np
import pytest

import workloads as W
from tests import gpu_cases as G

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def klr():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1911_02373_gb300 as k
    return k


@pytest.fixture(scope="module")
def setup(klr):
    ctx = klr.Context(0)
    gt = G.make_program(6, 48)
    prog = G.gpu_program(klr, torch.tensor(gt.coef.astype(np.float32)).cuda(), gt, torch)
    hw = klr.make_hw(W.HARDWARE)
    cfg = torch.tensor(klr.enumerate_configs(2)).cuda()
    return ctx, prog, hw, cfg


def _host(res):
    return [r.cpu().numpy() for r in res]


def _queries(sizes_per_kernel):
    off = np.concatenate([[0], np.cumsum([len(s) for s in sizes_per_kernel])]).astype(np.int64)
    return (torch.tensor(off).cuda(),
            torch.tensor(np.concatenate(sizes_per_kernel).astype(np.int64)).cuda())


def test_history_replays_argmin_bitwise(klr, setup):
    ctx, prog, hw, cfg = setup
    sizes = [W.log_spaced_sizes(64)] * 48
    qo, qn = _queries(sizes)
    ref = _host(ctx.argmin(prog, hw, cfg, qo, qn, out_dtype=klr.F32))
    hist = klr.History(ctx, 14)
    first = _host(klr.argmin_history(ctx, hist, prog, hw, cfg, qo, qn))
    for a, b in zip(first, ref):
        assert np.array_equal(a, b)
    assert not np.any(first[3] & klr.Q_HISTORY)
    second = _host(klr.argmin_history(ctx, hist, prog, hw, cfg, qo, qn))
    assert np.all(second[3] & klr.Q_HISTORY)
    assert np.array_equal(second[3] & ~klr.Q_HISTORY, first[3])
    for i in (0, 1, 2, 4):
        assert np.array_equal(second[i], first[i])
    hist.clear()
    third = _host(klr.argmin_history(ctx, hist, prog, hw, cfg, qo, qn))
    assert not np.any(third[3] & klr.Q_HISTORY)
    hist.close()


def test_history_mixed_hits_and_misses(klr, setup):
    ctx, prog, hw, cfg = setup
    rng = np.random.default_rng(3)
    old = [np.sort(rng.choice(2 ** np.arange(8, 24), 6, replace=False)) for _ in range(48)]
    hist = klr.History(ctx, 14)
    qo, qn = _queries(old)
    klr.argmin_history(ctx, hist, prog, hw, cfg, qo, qn)
    # kernel k now asks its old sizes again, new sizes (odd kernels only), and
    # one size twice
    new = []
    for k in range(48):
        s = list(old[k]) + ([int(old[k][0]) + 77, int(old[k][1]) * 3] if k % 2 else [])
        s.append(int(old[k][2]))
        new.append(np.array(s, dtype=np.int64))
    qo2, qn2 = _queries(new)
    got = _host(klr.argmin_history(ctx, hist, prog, hw, cfg, qo2, qn2))
    ref = _host(ctx.argmin(prog, hw, cfg, qo2, qn2, out_dtype=klr.F32))
    for i in (0, 1, 2, 4):
        assert np.array_equal(got[i], ref[i])
    assert np.array_equal(got[3] & ~klr.Q_HISTORY, ref[3])
    was_old = np.concatenate([np.isin(new[k], old[k]) for k in range(48)])
    assert np.array_equal((got[3] & klr.Q_HISTORY) != 0, was_old)
    # the answers are the oracle's (the usual argmin bar)
    gt = G.make_program(6, 48)
    o = G.oracle_choose(gt.coef.astype(np.float32), gt, qo2.cpu().numpy(), qn2.cpu().numpy())
    o["cycles"] = o["cycles"].reshape(len(got[0]), -1)
    o["boundary"] = o["boundary"].reshape(len(got[0]), -1)
    strict, _ = G.compare_argmin(got[0], got[1], o, 1e-4, 1e-6, 1e-5)
    assert strict > 0
    hist.close()


def test_full_history_loses_recordings_not_answers(klr, setup):
    ctx, prog, hw, cfg = setup
    sizes = [W.log_spaced_sizes(64)] * 48          # 3,072 keys, 1,024 slots
    qo, qn = _queries(sizes)
    ref = _host(ctx.argmin(prog, hw, cfg, qo, qn, out_dtype=klr.F32))
    hist = klr.History(ctx, 10)
    klr.argmin_history(ctx, hist, prog, hw, cfg, qo, qn)
    got = _host(klr.argmin_history(ctx, hist, prog, hw, cfg, qo, qn))
    hits = (got[3] & klr.Q_HISTORY) != 0
    assert 0 < hits.sum() <= 1024
    for i in (0, 1, 2, 4):
        assert np.array_equal(got[i], ref[i])
    with pytest.raises(klr.KlrError):
        klr.History(ctx, 40)
    hist.close()
