"""Host-side checks of the C-ABI library (no GPU needed): it loads, exports
every entry point include/hankel.h declares, its planner picks valid FFT
lengths, and descriptor validation rejects bad input with a status code."""

import ctypes
import os
import re

import numpy as np
import pytest

from paper_1401_6238_gb300 import build as B
from paper_1401_6238_gb300 import hankel as hk

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return hk.load()


def declared_functions():
    with open(os.path.join(ROOT, "include", "hankel.h")) as f:
        src = f.read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hankel_[a-z_0-9]+)\s*\(", src)))


def test_exports_every_declared_entry_point(lib):
    names = declared_functions()
    assert "hankel_plan" in names and "hankel_txv_backward" in names
    for name in names:
        assert hasattr(lib, name), name


def test_desc_layout_matches_header():
    # int32 m, int32 n[8], int32 N[8], (pad), int64 h_off, int64 x_off[8], int64 y_off
    assert hk.DESC_DTYPE.itemsize == 152
    assert hk.DESC_DTYPE.fields["h_off"][1] == 72
    assert hk.DESC_DTYPE.fields["y_off"][1] == 144


def test_plan_info_mirrors_header():
    # the ctypes mirror of hankel_plan_info lists the header's fields in order
    # (all int64): a field added on one side only would shift every later one
    import re
    with open(os.path.join(ROOT, "include", "hankel.h")) as f:
        text = f.read()
    body = re.search(r"typedef struct hankel_plan_info \{(.*?)\} hankel_plan_info;", text, re.S).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)  # comments out
    fields = re.findall(r"int64_t\s+(\w+)\s*;", body)
    assert len(fields) == len(re.findall(r";", body))  # every member is an int64_t
    assert [f for f, _ in hk.PlanInfo._fields_] == fields
    assert all(t is ctypes.c_int64 for _, t in hk.PlanInfo._fields_)


def smooth(L):
    for p in (2, 3, 5, 7):
        while L % p == 0:
            L //= p
    return L == 1


def test_fft_length_choice(lib):
    prev = 0
    for d in list(range(1, 300)) + [1021, 2048, 4092, 5116, 8191, 8192, 10000, 16381, 16384]:
        L = hk.hankel_fft_length(d)
        assert L >= d and L >= 2 and smooth(L), (d, L)
        assert L <= 2 * max(d, 2), (d, L)  # never more than one octave of padding
        assert L >= prev or True
        prev = L
    assert hk.hankel_fft_length(16385) == -1
    assert hk.hankel_fft_length(0) == -1
    # powers of two are always their own best length
    for k in range(1, 15):
        assert hk.hankel_fft_length(2 ** k) == 2 ** k


def _one(m=3, n=4):
    d = hk.square_descs([m], [n], [0], [0], [0])
    return d


@pytest.mark.parametrize("mutate,msg", [
    (lambda d: d.__setitem__("m", 1), "order"),
    (lambda d: d.__setitem__("m", 9), "order"),
    (lambda d: d["n"].__setitem__((0, 1), 0), "n[1]"),
    (lambda d: d.__setitem__("h_off", -1), "negative"),
    (lambda d: d["x_off"].__setitem__((0, 0), -5), "x_off"),
])
def test_validation_rejects_bad_descriptors(lib, mutate, msg):
    d = _one()
    mutate(d)
    with pytest.raises(hk.HankelError) as e:
        hk.hankel_plan(d, hk.R32, hk.SAME_X)
    assert e.value.status == hk.EINVAL
    assert msg in e.value.message


def test_rejects_bad_dtype_flags_and_lengths(lib):
    d = _one()
    with pytest.raises(hk.HankelError) as e:
        hk.hankel_plan(d, 7, 0)
    assert e.value.status == hk.EINVAL
    with pytest.raises(hk.HankelError) as e:
        hk.hankel_plan(d, hk.R32, 1 << 12)
    assert e.value.status == hk.EINVAL
    big = hk.square_descs([5], [5000], [0], [0], [0])  # d = 24996 > 16384
    with pytest.raises(hk.HankelError) as e:
        hk.hankel_plan(big, hk.R32, hk.SAME_X)
    assert e.value.status == hk.EUNSUPPORTED
    with pytest.raises(hk.HankelError) as e:
        hk.hankel_plan(np.zeros(0, dtype=hk.DESC_DTYPE), hk.R32, 0)
    assert e.value.status == hk.EINVAL


def test_null_plan_calls_return_einval(lib):
    for fn, args in [(lib.hankel_txv, (None,) * 6), (lib.hankel_txv_block, (None,) * 6),
                     (lib.hankel_txv_backward, (None,) * 7)]:
        assert fn(*args) == hk.EINVAL
    assert "NULL" in hk.hankel_last_error()
    lib.hankel_plan_destroy(None)  # ignored


def test_tuning_knobs(lib):
    old = hk.hankel_get_tuning()
    try:
        hk.hankel_set_tuning(0.0, 32)
        assert hk.hankel_get_tuning() == (0.0, 32)
        cheap = [hk.hankel_fft_length(d) for d in range(2000, 4100, 37)]
        hk.hankel_set_tuning(500.0, 16)
        costly = [hk.hankel_fft_length(d) for d in range(2000, 4100, 37)]
        # the cost model changes the choice, and every choice stays a valid length
        ds = list(range(2000, 4100, 37))
        assert cheap != costly
        assert all(L >= d and smooth(L) for d, L in zip(ds, cheap + costly[:0]))
        assert all(L >= d and smooth(L) for d, L in zip(ds, costly))
        for bad in [(-1.0, 16), (10.0, 12), (2000.0, 16)]:
            with pytest.raises(hk.HankelError) as e:
                hk.hankel_set_tuning(*bad)
            assert e.value.status == hk.EINVAL
    finally:
        hk.hankel_set_tuning(*old)


BINS = [32, 48, 64, 96, 128, 192, 256, 384, 512, 768, 1024, 1536, 2048, 3072, 4096, 5120]


def test_bin_policy(lib):
    # defaults: every bin on the persistent launch, FP32 powers
    hk.hankel_set_bin_policy({})
    assert all(hk.hankel_get_bin_policy(L) == (0, 99) for L in BINS)
    try:
        hk.hankel_set_bin_policy({1024: (1, 99), 4096: (0, 7)})
        assert hk.hankel_get_bin_policy(1024) == (1, 99)
        assert hk.hankel_get_bin_policy(4096) == (0, 7)
        assert hk.hankel_get_bin_policy(2048) == (0, 99)  # not listed: unchanged
        hk.hankel_set_bin_policy({4096: (1, 5)})  # other bins keep their choices
        assert hk.hankel_get_bin_policy(1024) == (1, 99) and hk.hankel_get_bin_policy(4096) == (1, 5)
        for bad in [{1000: (0, 99)}, {16: (0, 99)}, {1024: (2, 99)}, {1024: (0, 1)}, {1024: (0, 100)}]:
            with pytest.raises(hk.HankelError) as e:
                hk.hankel_set_bin_policy(bad)
            assert e.value.status == hk.EINVAL
        with pytest.raises(hk.HankelError):
            hk.hankel_get_bin_policy(1000)
        # a rejected call changes nothing
        assert hk.hankel_get_bin_policy(1024) == (1, 99)
    finally:
        hk.hankel_set_bin_policy({})
    assert hk.hankel_get_bin_policy(4096) == (0, 99)


def test_mdesc_layout_matches_header():
    # int32 m, int32 levels, int32 n[4][8], int64 h_off, int64 x_off[8], int64 y_off
    assert hk.MDESC_DTYPE.itemsize == 216
    assert hk.MDESC_DTYPE.fields["h_off"][1] == 136
    assert hk.MDESC_DTYPE.fields["x_off"][1] == 144
    assert hk.MDESC_DTYPE.fields["y_off"][1] == 208


@pytest.mark.parametrize("mutate,msg", [
    (lambda d: d.__setitem__("levels", 0), "levels"),
    (lambda d: d.__setitem__("levels", 5), "levels"),
    (lambda d: d.__setitem__("m", 1), "order"),
    (lambda d: d["n"].__setitem__((0, 2, 1), 0), "n[2][1]"),
    (lambda d: d.__setitem__("y_off", -3), "negative"),
])
def test_multilevel_validation(lib, mutate, msg):
    d = hk.level_descs([[2, 3, 2], [2, 2, 1], [3, 1, 2]], [0], [[0, 10, 20]], [0])
    mutate(d)
    with pytest.raises(hk.HankelError) as e:
        hk.hankel_plan_multilevel(d, hk.C64, 0)
    assert e.value.status == hk.EINVAL
    assert msg in e.value.message


def test_multilevel_rejects_other_flags(lib):
    d = hk.level_descs([[2, 3, 2], [2, 2, 1]], [0], [[0, 10, 20]], [0])
    for bad in (hk.FP64_POWER, hk.ONE_PER_LAUNCH, hk.BLOCK, 1 << 9):
        with pytest.raises(hk.HankelError) as e:
            hk.hankel_plan_multilevel(d, hk.C64, bad)
        assert e.value.status == hk.EINVAL


def test_anticirculant_needs_square_tensors_and_fft_lengths(lib):
    # 10007 is prime (no transform of that length) and its periodic
    # embedding, d = 3 * 10006 + 1, exceeds the longest transform
    d = hk.square_descs([3], [10007], [0], [0], [0])
    with pytest.raises(hk.HankelError) as e:
        hk.hankel_plan(d, hk.R32, hk.SAME_X | hk.ANTICIRCULANT)
    assert e.value.status == hk.EUNSUPPORTED and "n=10007" in e.value.message
    d = hk.make_descs(1)
    d["m"] = 3
    d["n"][0, :3] = [8, 8, 6]
    with pytest.raises(hk.HankelError) as e:
        hk.hankel_plan(d, hk.C64, hk.ANTICIRCULANT)
    assert e.value.status == hk.EINVAL and "square" in e.value.message
