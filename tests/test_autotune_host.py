"""Host logic of the persistent launch's autotuner (no GPU): which launch
shapes fit an SM's shared memory, that the fastest timed shape wins, and that
the choice is cached per code shape and batch-size bucket.  CUDA events and
device properties are replaced by fakes; the timed "launch" only advances a
fake clock by a programmed duration."""
import types

import pytest
import torch

from paper_1903_10107_gb300 import autotune


class FakeCode:
    def __init__(self, Mb, Nb, Z, edges, max_row_deg):
        self.Mb, self.Nb, self.Z = Mb, Nb, Z
        self.n, self.m = Nb * Z, Mb * Z
        self.edges, self.max_row_deg = edges, max_row_deg
        self.device = torch.device("cpu")


MIXED = FakeCode(24, 96, 512, 192000, 22)  # n = 49152: 192 KB of soft values per word
SMALL = FakeCode(8, 32, 128, 12288, 18)    # n = 4096
NARROW = FakeCode(256, 1024, 32, 98304, 12)  # n = 32768, Z = 32: one word, one CTA, 64 threads


@pytest.fixture
def fake_cuda(monkeypatch, tmp_path):
    props = types.SimpleNamespace(shared_memory_per_multiprocessor=228 * 1024,
                                  shared_memory_per_block_optin=227 * 1024)
    clock = {"t": 0.0}

    class Event:
        def __init__(self, enable_timing=False):
            self.t = None

        def record(self, stream=None):
            self.t = clock["t"]

        def elapsed_time(self, end):
            return end.t - self.t

    monkeypatch.setattr(torch.cuda, "get_device_properties", lambda dev=None: props)
    monkeypatch.setattr(torch.cuda, "current_stream", lambda dev=None: None)
    monkeypatch.setattr(torch.cuda, "synchronize", lambda dev=None: None)
    monkeypatch.setattr(torch.cuda, "Event", Event)
    monkeypatch.setattr(autotune, "_CACHE_PATH", str(tmp_path / "autotune.json"))
    return clock


def launcher(clock, ms, calls):
    def run(words, ctas, threads, n_frames):
        calls.append((words, ctas, threads, n_frames))
        clock["t"] += ms[(words, ctas, threads)]
    return run


def test_candidates_fit_shared_memory_and_registers(fake_cuda):
    # one word of the n = 49152 code's soft values is 192 KB: one CTA per SM, one word;
    # one thread pair per row of a layer (1024 threads) or half as many
    assert autotune.candidates(MIXED) == [(1, 1, 1024), (1, 1, 512)]
    c = autotune.candidates(SMALL)
    assert (1, 4, 256) in c and (2, 2, 512) in c and (4, 1, 1024) in c and (4, 2, 512) in c
    assert (2, 4, 512) not in c and (4, 2, 1024) not in c and (4, 3, 512) not in c  # registers
    for words, ctas, threads in c:
        per_cta = 4 * SMALL.n * words + SMALL.m * words
        assert ctas * per_cta <= 228 * 1024
        assert ctas * threads * 64 <= 65536
        assert threads % (32 * words) == 0


def test_default_threads_follow_the_rows_of_a_layer():
    assert autotune.default_threads(MIXED, 1) == 1024
    assert autotune.default_threads(SMALL, 1) == 256 and autotune.default_threads(SMALL, 4) == 1024
    wide = FakeCode(8, 80, 128, 30720, 40)  # rows of 40 edges: 20 slots per half row, 512 threads at most
    assert autotune.default_threads(wide, 4) == 512
    odd = FakeCode(4, 16, 13, 13 * 20, 6)
    assert autotune.default_threads(odd, 1) == 32  # 26 threads rounded up to a warp


def test_single_candidate_needs_no_timing(fake_cuda):
    calls = []
    assert autotune.candidates(NARROW) == [(1, 1, 64)]
    assert autotune.tune_persistent(NARROW, launcher(fake_cuda, {}, calls), 16384) == (1, 1, 64)
    assert calls == []


def test_headline_code_times_both_thread_counts(fake_cuda):
    calls = []
    ms = {(1, 1, 1024): 30.0, (1, 1, 512): 33.0}
    assert autotune.tune_persistent(MIXED, launcher(fake_cuda, ms, calls), 16384, sample_frames=4096) == (1, 1, 1024)
    assert {c[:3] for c in calls} == set(ms)
    calls.clear()
    ms = {(1, 1, 1024): 30.0, (1, 1, 512): 29.0}
    assert autotune.tune_persistent(MIXED, launcher(fake_cuda, ms, calls), 16384, force=True) == (1, 1, 512)


def test_fastest_shape_wins_and_is_cached(fake_cuda):
    cands = autotune.candidates(SMALL)
    ms = {c: 10.0 + i for i, c in enumerate(cands)}
    ms[(2, 2, 512)] = 1.0
    calls = []
    assert autotune.tune_persistent(SMALL, launcher(fake_cuda, ms, calls), 3000, sample_frames=1024) == (2, 2, 512)
    assert {c[:3] for c in calls} == set(cands)
    assert all(nf == 1024 for *_, nf in calls)  # timed on a sample of the batch
    # same code shape, same batch bucket (4096): cached, nothing launched
    calls.clear()
    ms2 = {**ms, (2, 2, 512): 50.0}
    assert autotune.tune_persistent(SMALL, launcher(fake_cuda, ms2, calls), 4000) == (2, 2, 512)
    assert calls == []
    # another bucket, or force, times again
    assert autotune.tune_persistent(SMALL, launcher(fake_cuda, ms2, calls), 5000) != (2, 2, 512)
    assert calls
    calls.clear()
    assert autotune.tune_persistent(SMALL, launcher(fake_cuda, ms2, calls), 4000, force=True) != (2, 2, 512)
    assert calls


def test_cache_key_separates_code_shapes():
    other = FakeCode(8, 32, 128, 12288, 20)
    assert autotune._key(SMALL, 4096) != autotune._key(other, 4096)
    assert autotune._key(SMALL, 3000) == autotune._key(SMALL, 4096) != autotune._key(SMALL, 4097)
