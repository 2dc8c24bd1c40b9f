"""The autotuner's search space (grom_tune_space, host arithmetic only) and the
binding's struct layouts against include/grom.h, compiled by gcc.  No GPU:
nothing here launches a kernel."""
import ctypes
import os
import subprocess

import pytest

import paper_2311_03694_gb300 as grom

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SM = 152


@pytest.fixture(scope="module", autouse=True)
def _lib():
    grom.build()
    grom.load()


def _key(e):
    return (e["kernel"], e["tile_m"], e["split_a"], e["split_b"])


def _k3t_split_max(n, rank, form, which):
    np_ = (n + 63) // 64 * 64
    rp = (rank + 63) // 64 * 64
    k = np_ if which == 1 else (2 if form == "cp_skew" else 1) * rp
    return max(1, (k // 64) // 4)


@pytest.mark.parametrize("form,storage,layout,rank", [
    ("full", "bf16", "dense", 0), ("full", "bf16", "skew_packed", 0),
    ("cp", "bf16", "dense", 96), ("cp_skew", "bf16", "dense", 1024)])
@pytest.mark.parametrize("batch", [1, 8, 9, 16, 17, 40, 130, 256, 1024])
def test_space_starts_with_the_rule_and_has_no_duplicates(form, storage, layout, rank, batch):
    n = 1024
    sp = grom.tune_space(form, storage, n, batch, max_batch=1024, rank=rank, layout=layout, sm_count=SM)
    assert all(e["batch"] == batch for e in sp)
    rule_tensor = batch > 8 if form == "full" else batch >= 16
    assert sp[0]["kernel"] == ("tensor" if rule_tensor else "stream")
    assert (sp[0]["tile_m"], sp[0]["split_a"], sp[0]["split_b"]) == (0, 0, 0)
    # the other family with its rule shape comes next
    assert sp[1]["kernel"] == ("stream" if rule_tensor else "tensor")
    assert (sp[1]["tile_m"], sp[1]["split_a"], sp[1]["split_b"]) == (0, 0, 0)
    keys = [_key(e) for e in sp]
    assert len(set(keys)) == len(keys)
    for e in sp[2:]:
        assert e["kernel"] == "tensor"
        if form == "full" and layout == "dense":
            assert e["tile_m"] == 0 and e["split_b"] == 0 and 1 <= e["split_a"] <= n
        elif form == "full":
            # every admissible height of the rule's kernel, then the other
            # kernel (1: single CTAs, 2: SM pairs) with its rule height
            assert e["split_a"] == 0
            assert (e["split_b"] == 0 and 8 <= e["tile_m"] <= 32) or (e["split_b"] in (1, 2) and e["tile_m"] == 0)
        else:
            assert e["tile_m"] == 0
            assert 1 <= e["split_a"] <= _k3t_split_max(n, rank, form, 1)
            assert 1 <= e["split_b"] <= _k3t_split_max(n, rank, form, 2)


@pytest.mark.parametrize("storage", ["f64", "f32x2", "f32"])
@pytest.mark.parametrize("form", ["full", "cp", "cp_skew", "svd"])
def test_no_tensor_kernel_no_alternatives(storage, form):
    # without BF16 storage (and for the SVD form) only the SIMT kernels exist
    sp = grom.tune_space(form, storage, 256, 64, rank=32, sm_count=SM)
    assert sp == [dict(sp[0])] and sp[0]["kernel"] == "stream"


def test_svd_bf16_has_no_tensor_kernel():
    sp = grom.tune_space("svd", "bf16", 256, 64, rank=32, sm_count=SM)
    assert len(sp) == 1 and sp[0]["kernel"] == "stream"


def test_packed_space_has_the_other_k2p_kernel():
    # n = 1024 (four 128-position blocks): SM pairs by the rule, so the space
    # offers single CTAs
    for batch, other in [(9, 1), (64, 1), (256, 1), (1024, 1)]:
        sp = grom.tune_space("full", "bf16", 1024, batch, max_batch=1024, layout="skew_packed", sm_count=SM)
        assert [e["split_b"] for e in sp if e["split_b"] != 0] == [other]
    # n = 200: one block, no pairs
    sp = grom.tune_space("full", "bf16", 200, 512, max_batch=512, layout="skew_packed", sm_count=SM)
    assert all(e["split_b"] == 0 for e in sp)


@pytest.mark.parametrize("form,layout,rank", [("full", "dense", 0), ("full", "skew_packed", 0), ("cp_skew", "dense", 512)])
def test_one_entry_serves_a_bucket(form, layout, rank):
    # batches with the same ceil(batch / 16) share every plan: same space
    for lo, hi in [(17, 32), (129, 144), (1009, 1024)]:
        a = grom.tune_space(form, "bf16", 1024, lo, max_batch=1024, rank=rank, layout=layout, sm_count=SM)
        b = grom.tune_space(form, "bf16", 1024, hi, max_batch=1024, rank=rank, layout=layout, sm_count=SM)
        assert [_key(e) for e in a] == [_key(e) for e in b]


def test_k2p_tile_heights_are_bounded_by_the_scratch():
    # lower tiles mean more tiles and a larger mirrored-entry scratch: the
    # heights admitted are the tallest ones, down to what create's scratch holds
    sp = grom.tune_space("full", "bf16", 1024, 40, max_batch=64, layout="skew_packed", sm_count=SM)
    sp = [e for e in sp if e["split_b"] == 0]  # the rule's kernel (single CTAs at 40 trajectories)
    ms = sorted(e["tile_m"] for e in sp[2:])
    assert len(ms) >= 8 and set(ms) <= set(range(8, 33))
    rule = (set(range(min(ms), 33)) - set(ms))
    assert len(rule) <= 1  # a contiguous range up to 32, less the rule's own height
    # a ROM sized for larger batches holds more scratch: more heights
    big = grom.tune_space("full", "bf16", 1024, 40, max_batch=1024, layout="skew_packed", sm_count=SM)
    assert {e["tile_m"] for e in sp[2:]} <= {e["tile_m"] for e in big[2:] if e["split_b"] == 0}


def test_larger_scratch_admits_more_splits():
    # K2's split count is bounded by the scratch create allocates for max_batch:
    # a ROM sized for bigger batches (smaller rule splits there, but larger
    # scratch) admits at least as many alternatives at a small batch
    small = grom.tune_space("full", "bf16", 512, 16, max_batch=16, sm_count=SM)
    large = grom.tune_space("full", "bf16", 512, 16, max_batch=1024, sm_count=SM)
    assert {_key(e) for e in small} <= {_key(e) for e in large}


@pytest.mark.parametrize("args", [
    ("full", "bf16", 0, 1), ("full", "bf16", 64, 0), ("full", "bf16", 64, 65),
    ("cp", "bf16", 64, 1), ("svd", "f64", 64, 1)])
def test_invalid_arguments(args):
    form, storage, n, batch = args
    with pytest.raises(grom.GromError):
        grom.tune_space(form, storage, n, batch, max_batch=64, rank=0, sm_count=SM)


def test_deterministic():
    a = grom.tune_space("cp_skew", "bf16", 1024, 256, max_batch=1024, rank=1024, sm_count=SM)
    b = grom.tune_space("cp_skew", "bf16", 1024, 256, max_batch=1024, rank=1024, sm_count=SM)
    assert a == b and len(a) > 2


def _c_layout(struct, fields, tmp_path):
    src = tmp_path / "layout.c"
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "grom.h"', "int main(void) {",
             '  printf("%%zu\\n", sizeof(%s));' % struct]
    lines += ['  printf("%%zu\\n", offsetof(%s, %s));' % (struct, f) for f in fields]
    lines += ["  return 0;", "}"]
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-I" + os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    return [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]


@pytest.mark.parametrize("cls,struct", [
    (grom._Tuning, "grom_tuning"), (grom._Desc, "grom_desc"), (grom._Request, "grom_request"),
    (grom._Result, "grom_result"), (grom._Stats, "grom_serve_stats")])
def test_binding_structs_match_the_header(cls, struct, tmp_path):
    names = [f[0] for f in cls._fields_]
    got = _c_layout(struct, names, tmp_path)
    assert got[0] == ctypes.sizeof(cls)
    assert got[1:] == [getattr(cls, f).offset for f in names]


class _FakeRom:
    """Stands in for a Rom in the cache logic: autotune returns a fixed entry
    per batch, set_tuning records what is installed."""

    form, storage, layout, n, rank, max_batch = "full", "bf16", "skew_packed", 512, 0, 1024

    def __init__(self, tile_m=0):
        self.tile_m = tile_m
        self.installed = []

    def autotune(self, batch, reps=0):
        return {"batch": batch, "kernel": "tensor", "tile_m": self.tile_m, "split_a": 0, "split_b": 0, "timed": 3,
                "ms": 1.0, "ms_rule": 1.0}

    def set_tuning(self, e):
        self.installed.append(e)


def test_tuning_cache_merges_per_bucket_and_reapplies(tmp_path):
    from paper_2311_03694_gb300 import tune

    path = str(tmp_path / "cache.json")
    tune.tune(_FakeRom(20), [16, 64], SM, path=path)
    # a later run for a batch of the same bucket as 64 replaces that entry
    tune.tune(_FakeRom(24), [60, 256], SM, path=path)
    rom = _FakeRom()
    assert tune.apply(rom, SM, path) == 3
    assert [(e["batch"], e["tile_m"]) for e in rom.installed] == [(16, 20), (60, 24), (256, 24)]
    # another device (SM count) or ROM shape has its own key
    assert tune.apply(_FakeRom(), SM - 4, path) == 0
    other = _FakeRom()
    other.n = 256
    assert tune.apply(other, SM, path) == 0
