"""The batched engine's autotuner (``autotune.BatchTuner``), on the CPU with a
fake timer: which candidate it keeps, what it times (a stratified sample of the
batch, compiled by the real host compiler), and that a second batch of the same
kind reuses the cached choice without timing again."""
import numpy as np
import pytest

from paper_2308_01999_gb300 import inputs as gen


@pytest.fixture(scope="module")
def mods():
    from paper_2308_01999_gb300 import _build
    _build.build()
    from paper_2308_01999_gb300 import autotune, sv
    sv.lib()
    return autotune, sv


def _states(count, seed, nmin=10, nmax=16):
    work = gen.batched_ansatz_workload(count=count, nmin=nmin, nmax=nmax, seed=seed)
    return [(n, g, p) for n, g, p, _ in work]


def test_keeps_the_fastest_candidate_and_caches_it(mods):
    autotune, sv = mods
    calls = []

    def fake_timer(sub, fw, win, keep, tile):
        calls.append((fw, win, keep, tile, len(sub.ns)))
        b = sv.Batch(None)                    # the sample really compiles
        b.compile(sub, fw, win, bool(keep), tile)
        b.close()
        return {(3, 4, 1, 14): 1.0, (1, 0, 0, 14): 1.5}.get((fw, win, keep, tile), 2.0 + 0.1 * fw)

    tuner = autotune.BatchTuner(fake_timer, sample=40)
    packed = sv.pack_batch(_states(120, 1))
    assert tuner.choose(packed) == (3, 4, 1, 14)
    assert [c[:4] for c in calls] == list(autotune.CANDIDATES)
    assert all(c[4] == 40 for c in calls)
    # another batch of the same kind: cached, nothing timed
    again = sv.pack_batch(_states(90, 2))
    assert autotune.signature(again.ns, again.gate_counts) == autotune.signature(packed.ns, packed.gate_counts)
    assert tuner.choose(again) == (3, 4, 1, 14) and len(calls) == len(autotune.CANDIDATES)
    # a batch of another kind (other qubit range) is timed anew
    other = sv.pack_batch(_states(30, 3, nmin=5, nmax=8))
    tuner.choose(other)
    assert len(calls) == 2 * len(autotune.CANDIDATES)


def test_ties_go_to_the_earlier_candidate_and_rejected_options_are_skipped(mods):
    autotune, sv = mods

    def timer(sub, fw, win, keep, tile):
        if fw == 1:
            raise sv.SvError(2, "rejected")
        return 5.0

    tuner = autotune.BatchTuner(timer, sample=8)
    assert tuner.choose(sv.pack_batch(_states(20, 4))) == (2, 4, 0, 14)


def test_stratified_sample_keeps_the_size_mix(mods):
    autotune, _ = mods
    rng = np.random.default_rng(0)
    ns = [int(x) for x in rng.integers(10, 21, size=4096)]
    idx = autotune.stratified_sample(ns, 512)
    assert len(idx) == 512 and len(set(idx)) == 512
    full = np.bincount(ns, minlength=21)[10:] / len(ns)
    samp = np.bincount([ns[i] for i in idx], minlength=21)[10:] / len(idx)
    assert np.max(np.abs(full - samp)) < 0.01
    assert autotune.stratified_sample(ns[:5], 10) == [0, 1, 2, 3, 4]


def test_batch_compile_uses_the_tuner(mods):
    autotune, sv = mods
    tuner = autotune.BatchTuner(
        lambda sub, fw, win, keep, tile: float((fw, win, keep, tile) == (2, 3, 0, 12)) * -1.0 + 1.0, sample=16)
    b = sv.Batch(None)
    b.compile(_states(50, 5), tuner=tuner)
    assert b.choice == (2, 3, 0, 12)
    b.close()
