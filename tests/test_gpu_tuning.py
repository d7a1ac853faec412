"""Launch configurations and the autotuner: every candidate configuration must
give bit-identical results; the tuner must return a configuration from the
candidate sets and leave results unchanged."""
import numpy as np
import pytest

import tpcgen

pytestmark = pytest.mark.gpu

COMMON = {"ca_blocks_per_sm": [4, 8, 16], "elem_blocks_per_sm": [4, 8, 16], "fit_threads": [32, 64, 128],
          "fit_blocks_per_sm": [16, 32, 64]}
COMMON_DEFAULT = {"ca_blocks_per_sm": 8, "elem_blocks_per_sm": 8, "fit_threads": 64, "fit_blocks_per_sm": 32}
# finder launch shapes: the two-pass finder's unit CTAs (default), the fused finder's window CTAs
FINDERS = {0: ({"find_threads": [128, 256], "find_ctas_per_sm": [4, 8]}, {"find_threads": 128, "find_ctas_per_sm": 8}),
           8: ({"find_threads": [256, 384, 512], "find_ctas_per_sm": [1, 2]},
               {"find_threads": 384, "find_ctas_per_sm": 2})}


@pytest.fixture(scope="module")
def lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2208_07412_b300 import tpc
    tpc.load()
    return tpc


@pytest.fixture(scope="module")
def tf():
    return tpcgen.generate(tpcgen.full_tpc(5, n_tracks=3000))


def same(a, b):
    assert a["clusters"].tobytes() == b["clusters"].tobytes()
    assert a["tracks"].tobytes() == b["tracks"].tobytes()
    for k in ("up", "down", "chain_of", "cl2trk"):
        assert np.array_equal(a[k], b[k]), k


@pytest.mark.parametrize("flags", sorted(FINDERS))
def test_every_candidate_gives_identical_results(lib, tf, flags):
    cand, dflt = FINDERS[flags]
    CANDIDATES, DEFAULT = {**cand, **COMMON}, {**dflt, **COMMON_DEFAULT}
    with lib.Reconstructor.for_timeframe(tf, flags=flags) as R:
        assert lib.tpc_get_tuning(R.ctx) == DEFAULT
        ref = R.run(tf)
        for knob, values in CANDIDATES.items():
            for v in values:
                lib.tpc_set_tuning(R.ctx, **{knob: v})
                same(R.run(tf), ref)
            lib.tpc_set_tuning(R.ctx, **{knob: DEFAULT[knob]})
        with pytest.raises(lib.TpcError):
            lib.tpc_set_tuning(R.ctx, find_threads=300)
        other = FINDERS[8 - flags][1]["find_ctas_per_sm"]   # the other finder's shape is refused
        with pytest.raises(lib.TpcError):
            lib.tpc_set_tuning(R.ctx, find_ctas_per_sm=other)
        assert lib.tpc_get_tuning(R.ctx) == DEFAULT


@pytest.mark.parametrize("flags", sorted(FINDERS))
def test_autotune_picks_candidates_and_keeps_results(lib, tf, flags):
    CANDIDATES = {**FINDERS[flags][0], **COMMON}
    with lib.Reconstructor.for_timeframe(tf, flags=flags) as R:
        ref = R.run(tf)
        cfg = lib.tpc_autotune(R.ctx, tf.pages, tf.page_offsets, tf.n_time_bins, reps=2)
        assert set(cfg) == set(CANDIDATES)
        for k, v in cfg.items():
            assert v in CANDIDATES[k], (k, v)
        assert lib.tpc_get_tuning(R.ctx) == cfg
        same(R.run(tf), ref)
        # a busy context refuses to tune
        t = R.submit(tf.pages, tf.page_offsets, tf.n_time_bins)
        with pytest.raises(lib.TpcError) as ei:
            lib.tpc_autotune(R.ctx, tf.pages, tf.page_offsets, tf.n_time_bins)
        assert ei.value.code == -3
        R.wait(t)
        lib.tpc_release(R.ctx, t)
