"""CPU checks of the C-ABI library: it builds, loads without a GPU, exports
every symbol include/tilegs.h declares, and its host-only helpers (defaults,
layouts, argument checks) behave.  No kernel is launched here."""
import ctypes as C
import json
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "tilegs.h")


@pytest.fixture(scope="module")
def G():
    from paper_2609_03613_gb300 import build as B, tilegs
    B.build()
    tilegs.lib()
    return tilegs


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\**\s+(gs_[a-z_0-9]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_hot_path_calls():
    names = declared_functions()
    for n in ["gs_project", "gs_tile_intersect", "gs_sort_or_bin", "gs_rasterize_fwd", "gs_render"]:
        assert n in names


def test_library_exports_every_declared_symbol(G):
    lib = C.CDLL(G.LIB_PATH)
    names = declared_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(names) == sorted(G.EXPORTS)


def header_constants():
    """Every `GS_NAME = value` enumerator include/tilegs.h declares."""
    src = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    return {m.group(1): int(m.group(2)) for m in re.finditer(r"\b(GS_[A-Z0-9_]+)\s*=\s*(\d+)", src)}


def test_binding_constants_match_header(G):
    """The binding passes flags, modes and status codes as plain integers:
    each must be the header's value."""
    h = header_constants()
    for name in ["RENDER_HOST_INPUTS", "RENDER_HOST_OUTPUTS", "RENDER_NO_SYNC", "RENDER_GRAPH", "RENDER_SAVE",
                 "RENDER_PIPELINE", "MODE_GLOBAL_SORT", "MODE_BINNED_EXACT", "MODE_BINNED_PAPER",
                 "MODE_BINNED_NOREPAIR"]:
        assert getattr(G, name) == h["GS_" + name], name
    flags = [h[k] for k in h if k.startswith("GS_RENDER_")]
    assert len(set(flags)) == len(flags) and all(f & (f - 1) == 0 for f in flags)  # distinct single bits
    assert G.GS_OK == h["GS_OK"]
    errs = {v: k for k, v in h.items() if k.startswith("GS_ERR_")}
    assert sorted(G.ERRORS) == sorted(errs)
    assert G.MODES == {"global": h["GS_MODE_GLOBAL_SORT"], "exact": h["GS_MODE_BINNED_EXACT"],
                       "paper": h["GS_MODE_BINNED_PAPER"], "norepair": h["GS_MODE_BINNED_NOREPAIR"]}


def test_defaults_match_paper_tables(G):
    gold = json.load(open(os.path.join(ROOT, "tests", "golden", "paper_defaults.json")))
    cfg = G.default_config("paper")
    assert cfg.K == gold["K"]
    assert cfg.sample_count == gold["sample_count"]
    assert cfg.p_lo == pytest.approx(gold["p_lo"]) and cfg.p_hi == pytest.approx(gold["p_hi"])
    assert cfg.pad == pytest.approx(gold["pad"])
    assert cfg.near_alpha == pytest.approx(gold["near_alpha"])
    assert cfg.near_gamma == pytest.approx(gold["near_gamma"])
    assert cfg.eps == pytest.approx(gold["eps"])
    assert cfg.repair_budget_frac == pytest.approx(gold["repair"]["budget_frac"])
    assert cfg.near_shift == 1 and cfg.tile_size == 16
    assert G.default_config("exact").near_shift == 0
    # frame kernels launched with programmatic dependent launch by default
    assert G.default_config("exact").pdl == 1 and G.default_config("global").pdl == 1


def test_host_layout_helpers(G):
    L = G.lib()
    n = 1001
    offs = [L.gs_projected_offset(n, f) for f in range(6)]
    assert all(o % 256 == 0 for o in offs)
    assert offs[1] - offs[0] >= 16 * n and offs[4] - offs[3] >= 8 * n
    assert L.gs_projected_bytes(n) == offs[5]
    assert L.gs_isect_offset(77, 2) >= 2 * 77 * 4 and L.gs_isect_bytes(77) >= 3 * 77 * 4
    assert L.gs_num_tiles(1920, 1080, 16) == 120 * 68
    assert L.gs_num_tiles(250, 131, 16) == 16 * 9
    assert L.gs_num_tiles(0, 10, 16) == 0


def test_invalid_config_rejected_before_any_cuda_call(G):
    L = G.lib()
    for bad in (dict(K=0), dict(K=G.MAX_K + 1), dict(tile_size=12), dict(sample_count=9000),
                dict(mode=7), dict(pdl=2), dict(pdl=-1)):
        cfg = G.default_config("exact")
        for k, v in bad.items():
            setattr(cfg, k, v)
        h = C.c_void_p()
        assert L.gs_create(C.byref(h), C.byref(cfg)) == 1, bad
    cfg = G.default_config("exact")
    cfg.near_shift = 1
    h = C.c_void_p()
    assert L.gs_create(C.byref(h), C.byref(cfg)) == 1
    assert L.gs_status_string(2) == b"entry capacity exceeded"


def test_product_path_does_not_reference_the_oracle():
    pkg = os.path.join(ROOT, "paper_2609_03613_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "liboracle" not in txt, f
