"""GPU checks that the kernel choices of the tuning knobs never change a
result: each TCF bulk path (per-block and tiled, several tile targets) and
each GQF region bound leaves the oracle's table byte for byte, with the
oracle's statuses, after every insert and remove batch."""
import numpy as np
import pytest

from paper_2212_09005_gb300 import workloads as W
from gpu_util import dev_u64, zeros_u8, host, first_diff

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gf():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2212_09005_gb300 as gf

    gf.lib()
    return gf


def tcf_batches(lg, seed):
    n = int(0.75 * (1 << lg))
    keys = W.uniform_keys(seed, n)
    cuts = [0, 3, n // 9, n // 2, n]
    ins = [np.concatenate([keys[a:b], keys[a:a + (b - a) // 5]]) for a, b in zip(cuts, cuts[1:])]
    dels = [keys[: n // 4], np.concatenate([keys[n // 4: n // 2], W.uniform_keys(seed + 1, 1000)])]
    return ins, dels


@pytest.mark.parametrize("path,target", [(1, 0), (2, 128), (2, 512), (2, 1024)])
@pytest.mark.parametrize("lg,f", [(16, 16), (19, 16), (17, 8)])
def test_tcf_paths_leave_the_oracle_table(gf, oracle, path, target, lg, f):
    ins, dels = tcf_batches(lg, 3100 + lg)
    O = oracle.TCF(lg, f, seed=lg)
    G = gf.TCF(lg, f, gf.MODE_BULK, seed=lg, max_batch=max(map(len, ins + dels)))
    G.set_tuning(tcf_path=path, tcf_tile_target=target)
    assert G.get_tuning()["tcf_path"] == path
    for k, (b, op) in enumerate([(b, "insert") for b in ins] + [(b, "remove") for b in dels]):
        want = getattr(O, op)(b)
        st = zeros_u8(len(b))
        getattr(G, op)(dev_u64(b), st)
        assert np.array_equal(host(st), want), (op, k)
        d = first_diff(G.export(), O.export())
        assert d is None, (op, k, d)


def test_tcf_group_paths_agree(gf):
    """A TCF group under each path gives the same member tables."""
    import torch

    logs = [12, 14, 13, 15]
    imgs = []
    for path in (1, 2):
        T = gf.FilterGroup(gf.FILTER_TCF, logs, 16, [5, 6, 7, 8], max_total=1 << 16)
        T.set_tuning(tcf_path=path, tcf_tile_target=256)
        ks = [W.uniform_keys(3300 + m, int(0.85 * (1 << lg))) for m, lg in enumerate(logs)]
        off = torch.tensor(np.cumsum([0] + [len(k) for k in ks]), dtype=torch.int64, device="cuda")
        st = zeros_u8(int(off[-1]))
        T.insert(off, dev_u64(np.concatenate(ks)), st)
        imgs.append([T.export(m) for m in range(len(logs))] + [host(st)])
    for a, b in zip(*imgs):
        assert first_diff(a, b) is None


@pytest.mark.parametrize("groups", [1, 3, 8, 64])
def test_gqf_region_bound_leaves_the_oracle_table(gf, oracle, groups):
    q = 16
    keys = W.zipf_keys(3400, int(0.85 * (1 << q)), 1.2, 1 << 14)  # repeated keys: counters in the table
    O = oracle.GQF(q, 8, seed=4)
    G = gf.GQF(q, 8, seed=4, max_batch=len(keys))
    G.set_tuning(gqf_region_groups=groups)
    for b, op in [(keys[:5], "insert"), (keys[5: len(keys) // 3], "insert"), (keys[len(keys) // 3:], "insert"),
                  (keys[: len(keys) // 2], "remove"), (keys[::7], "remove")]:
        want = getattr(O, op)(b)
        st = zeros_u8(len(b))
        getattr(G, op)(dev_u64(b), st)
        assert np.array_equal(host(st), want), op
        d = first_diff(G.export(), O.export())
        assert d is None, (op, d)


def test_invalid_tuning_is_refused(gf):
    G = gf.TCF(12, 16, gf.MODE_BULK, seed=1)
    before = G.get_tuning()
    for bad in ({"tcf_path": 3}, {"tcf_tile_target": 64}, {"tcf_tile_target": 4096}, {"gqf_region_groups": 1000}):
        with pytest.raises(gf.FilterError):
            G.set_tuning(**bad)
    with pytest.raises(gf.FilterError):
        G.set_tuning(no_such_knob=1)
    assert G.get_tuning() == before
