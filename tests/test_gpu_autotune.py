"""The autotuner of the batched rollout's launch shape (threads per CTA x plan samples staged
per step) and its cache.

Every shape runs the same Alg. 1 rollout: the scanner warps only share out the plan samples
differently and the per-action maxima (or fixed-point sums) do not depend on the order, so
batched FCFS must give bit-identical results under each candidate shape, tuned or not.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2008_03518_gb300 import scenarios as S  # noqa: E402
from paper_2008_03518_gb300.fmdp import FmdpError, Scheduler  # noqa: E402

from test_gpu_batch import same_results, same_tables, table_of  # noqa: E402

THREADS = (128, 192, 256, 320, 384)
STAGE = (512, 1024, 1536, 2048)


@pytest.fixture(scope="module")
def crowded():
    sc = S.crowded_batch(seed=121, n_requests=40)
    with Scheduler.from_scenario(sc) as s:
        res = s.schedule_many(sc.requests)
        tab = table_of(s)
    return sc, res, tab


@pytest.mark.parametrize("threads,stage", [(128, 512), (192, 1024), (256, 2048), (320, 1536), (384, 512)])
def test_every_shape_gives_the_sequential_results(crowded, threads, stage):
    sc, alone, t_alone = crowded
    with Scheduler.from_scenario(sc, batch_size=16, threads_per_cta=threads, index_stage_items=stage) as s:
        res = s.schedule_batch(sc.requests)
        st = s.stats()
        t = table_of(s)
    assert st["threads_per_cta"] == threads
    same_results(alone, res)
    same_tables(t_alone, t)


def test_small_staging_reads_the_overflow_from_the_index():
    """A staging buffer far smaller than the samples near a state: the rest are read from
    the index in global memory, with the same results."""
    sc = S.c2_plain_scale(n_requests=12)
    with Scheduler.from_scenario(sc) as s:
        alone = s.schedule_many(sc.requests)
    with Scheduler.from_scenario(sc, threads_per_cta=192, index_stage_items=64) as s:
        res = s.schedule_batch(sc.requests)
    same_results(alone, res)


def test_autotune_picks_a_candidate_caches_it_and_batches_use_it(crowded):
    sc, alone, t_alone = crowded
    with Scheduler.from_scenario(sc, batch_size=16) as s:
        rep = s.autotune(sc.requests)
        ch = rep["chosen"]
        # waves of 16 and 8 rollouts, every shape whose staging fits in shared memory
        assert rep["from_cache"] == 0 and rep["entries"] == 2
        assert 2 * len(THREADS) * (len(STAGE) - 1) <= rep["candidates"] <= 2 * len(THREADS) * len(STAGE)
        assert rep["sample"] == 16
        assert ch["threads_per_cta"] in THREADS and ch["index_stage_items"] in STAGE
        assert 0 < ch["ms"] <= rep["default_ms"]  # the default shape is one of the candidates
        assert rep["ctas_per_sm"] >= 1
        assert ch["n_actions"] == len(sc.actions) and ch["combine"] == 0
        assert ch["plans_bucket"] == int(len(sc.plans)).bit_length() and ch["wave_bucket"] == 5
        again = s.autotune(sc.requests)
        assert again["from_cache"] == 1 and again["candidates"] == 0 and again["chosen"] == ch
        # tuning admitted nothing
        assert len(s.query_plans(-(1 << 40), 1 << 40)) == len(sc.plans)
        shapes = {e["threads_per_cta"] for e in s.tune_cache()}
        assert len(s.tune_cache()) == 2
        s.snapshot()
        res_p = s.schedule_batch(sc.requests)  # pipelined: one CTA per SM, the widest shape
        st_p = s.stats()
        t_p = table_of(s)
        s.restore()
        s.set_batch_mode(1)  # waves: the tuned shapes
        res = s.schedule_batch(sc.requests)
        st = s.stats()
        t = table_of(s)
    assert st_p["threads_per_cta"] == 384
    assert st["threads_per_cta"] in shapes  # the last wave's tuned shape
    same_results(alone, res_p)
    same_tables(t_alone, t_p)
    same_results(alone, res)
    same_tables(t_alone, t)


def test_cache_round_trip_and_rejected_entries(crowded):
    sc = crowded[0]
    with Scheduler.from_scenario(sc, batch_size=16) as s:
        s.autotune(sc.requests[:8])
        entries = s.tune_cache()
    assert len(entries) == 1
    e = dict(entries[0])
    e["threads_per_cta"] = 192 if e["threads_per_cta"] != 192 else 256
    with Scheduler.from_scenario(sc, batch_size=16, batch_mode=1) as s:  # waves take the cached shape
        s.load_tune_cache([e])
        rep = s.autotune(sc.requests[:8])
        assert rep["from_cache"] == 1 and rep["chosen"]["threads_per_cta"] == e["threads_per_cta"]
        s.schedule_batch(sc.requests[:8])
        assert s.stats()["threads_per_cta"] == e["threads_per_cta"]
        bad = dict(e, threads_per_cta=100)
        with pytest.raises(FmdpError):
            s.load_tune_cache([bad])
        with pytest.raises(FmdpError):
            s.load_tune_cache([dict(e, index_stage_items=777)])


def test_explicit_options_take_precedence_over_the_cache(crowded):
    sc = crowded[0]
    with Scheduler.from_scenario(sc, batch_size=16, threads_per_cta=256) as s:
        rep = s.autotune(sc.requests[:8])
        s.schedule_batch(sc.requests[:8])
        assert s.stats()["threads_per_cta"] == 256
        assert rep["chosen"]["threads_per_cta"] in THREADS


def test_autotune_needs_the_index():
    sc = S.c1_plain_small()
    with Scheduler.from_scenario(sc, full_scan=True) as s:
        with pytest.raises(FmdpError):
            s.autotune(sc.requests[:4])
