"""CPU checks of the C ABI: the library loads, exports every function the
header declares, and its host-only planning agrees with the paper's printed
numbers and with the oracle's tiling."""
import ctypes
import json
import os
import re

import pytest

from oracle import method as M

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GOLD = os.path.join(ROOT, "tests", "golden")


@pytest.fixture(scope="module")
def di():
    from paper_2401_06744_gb300 import build as b

    b.build()
    import paper_2401_06744_gb300 as di

    di.load()
    return di


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(di_[a-z0-9_]+)\s*\(", txt))
    return names


def test_library_exports_every_declared_symbol(di):
    lib = ctypes.CDLL(di.LIB_PATH)
    declared = _declared()
    assert "di_inpaint" in declared and "di_oras_iteration" in declared
    for name in declared:
        assert hasattr(lib, name), name
    assert declared <= set(di.exported_symbols()), declared - set(di.exported_symbols())


def test_status_strings(di):
    assert di.status_string(di.OK) == "ok"
    assert di.status_string(di.EMPTY_MASK) == "empty mask"


def test_plan_matches_paper_constants(di):
    g = json.load(open(os.path.join(GOLD, "paper_constants.json")))
    p = di.plan(g["width"], g["height"], g["channels"], block=g["block"], overlap=g["overlap"])
    assert p["local_problems"] == g["local_problems"]
    assert p["levels"] == g["levels"]


@pytest.mark.parametrize("w,h,B,o", [(1, 1, 32, 6), (3840, 2160, 32, 6), (1280, 720, 16, 4),
                                     (333, 171, 8, 2), (77, 1, 8, 1), (60, 60, 32, 6)])
def test_plan_matches_oracle_tiling(di, w, h, B, o):
    p = di.plan(w, h, 2, block=B, overlap=o)
    assert p["levels"] == M.num_levels(h, w, B)
    lw, lh = w, h
    for l in range(p["levels"]):
        assert p["sizes"][l] == (lw, lh)
        assert p["blocks"][l] == (len(M.axis_blocks(lw, B, o)), len(M.axis_blocks(lh, B, o)))
        lh, lw = M.coarse_shape(lh, lw)


@pytest.mark.parametrize("kw", [dict(block=12), dict(block=8, overlap=5), dict(alpha=-1.0),
                                dict(downsample=3), dict(stop_rule=7),
                                dict(min_cycles=5, max_cycles=2), dict(refine_fp64=2),
                                dict(local_iters_cascade=-1),
                                # the 16-bit modes store the coarse levels narrow: 32x32
                                # blocks and the block smoother only
                                dict(precision=1, block=16), dict(precision=2, smoother=1)])
def test_plan_rejects_bad_config(di, kw):
    with pytest.raises(di.DiError):
        di.plan(64, 64, 1, **kw)


def test_plan_rejects_bad_sizes(di):
    for args in [(0, 5, 1), (5, 0, 1), (5, 5, 0), (5, 5, 5)]:
        with pytest.raises(di.DiError):
            di.plan(*args)


def test_plan_counts_narrow_coarse_storage(di):
    # 16-bit modes: the coarse levels' u[0], u[1] and r take 2 bytes per value
    p32 = di.plan(3840, 2160, 3)
    p16 = di.plan(3840, 2160, 3, precision=1)
    coarse = sum(w * h for (w, h) in p32["sizes"][1:]) * 3
    slack = 3 * 256 * p32["levels"]  # per-buffer alignment
    assert abs(p32["workspace_bytes"] - p16["workspace_bytes"] - 3 * 2 * coarse) <= slack
