"""Seeded random intervals and tunings against the oracle, bit for bit: segment sizes
l = 5..20, magnitudes 1 .. 1e17, lengths from one word to 2^22 bits, and every tuning
parameter drawn from its valid range (tiles 2^12..2^20, 1..13 pre-sieve groups,
medium / large thresholds, scatter groups and epochs)."""
import pytest

import oracle
from paper_1111_3297_gb300 import sieve as S
from paper_1111_3297_gb300 import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1111_3297_gb300 import build
    build.build_library()
    c = S.sieve_init(0, max_v=2 * 10**17 + (1 << 30))
    yield c
    c.close()


def draw(seed):
    r = workloads.SplitMix64(0x5EED + seed)
    l = 5 + r.below(16)
    mag = 10 ** (r.below(18))
    n = 1 + r.below(max(1, (1 << 22) >> l))
    f = (mag // (2 << l)) + r.below(1 << 10)
    tl = 12 + r.below(9)
    tune = dict(tile_log2=tl, presieve_groups=1 + r.below(13), coop_max=1 << (6 + r.below(8)),
                medium_max=1 << (8 + r.below(14)), window_tiles=1 << r.below(11), epoch_tiles=0)
    while (tune["window_tiles"] << tl) > (1 << 30):
        tune["window_tiles"] >>= 1
    tune["epoch_tiles"] = tune["window_tiles"] * (1 + r.below(8))
    return l, f, n, tune


@pytest.mark.parametrize("seed", range(40))
def test_random_interval_and_tuning(ctx, seed):
    l, f, n, tune = draw(seed)
    saved = [S.sieve_get_tuning(ctx, k) for k in range(4)]
    try:
        for k in range(4):
            S.sieve_set_tuning(ctx, k, **tune)
        out = torch.empty((n << l) // 32, dtype=torch.int32, device="cuda")
        S.sieve_segments(ctx, l, f, n, out)
        S.sieve_sync(ctx)
        got = out.cpu().numpy().view("uint32")
    finally:
        for k in range(4):
            S.sieve_set_tuning(ctx, k, **saved[k])
    want = oracle.sieve(l, f, n)
    assert (got == want).all(), (l, f, n, tune)
