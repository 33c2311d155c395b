"""CPU checks of the C-ABI boundary: the library builds, loads and exports every
function that include/bc.h declares (no compute calls: no GPU here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "bc.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_\s\*]*?\b(bc_[a-z_0-9]+)\s*\(", text, flags=re.M)
    return sorted(set(n for n in names if not n.endswith("_fn")))


def test_header_parses():
    fns = declared_functions()
    for must in ("bc_graph_create", "bc_compute", "bc_batch_submit", "bc_poll", "bc_debug_source",
                 "bc_status_string", "bc_last_error", "bc_set_allocator"):
        assert must in fns


def test_library_builds_and_exports_every_declared_symbol():
    from paper_2305_03317_b300 import build
    lib_path = build.build()
    lib = ctypes.CDLL(lib_path)
    missing = [f for f in declared_functions() if not hasattr(lib, f)]
    assert not missing, missing


def test_status_strings_without_gpu():
    import paper_2305_03317_b300 as bc
    lib = bc.load()
    assert bc.status_string(bc.BC_OK) == "BC_OK"
    assert bc.status_string(bc.BC_E_TIMEOUT) == "BC_E_TIMEOUT"
    # argument validation happens before any device work
    assert lib.bc_graph_create(None, None, 3, 0, 1, None, ctypes.byref(ctypes.c_void_p())) == bc.BC_E_INVALID_ARG
    assert "NULL" in bc.last_error()
    assert lib.bc_server_config(0, 0) == bc.BC_E_INVALID_ARG
    assert lib.bc_poll(12345) == bc.BC_E_INVALID_ARG


def test_product_path_has_no_oracle_import():
    pkg = os.path.join(ROOT, "paper_2305_03317_b300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                src = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle\b", src, flags=re.M), f
                assert "liboracle" not in src and "brandes.c" not in src, f


def test_tuning_cache_roundtrip_without_gpu(tmp_path):
    import paper_2305_03317_b300 as bc
    p = tmp_path / "tune.json"
    bc.tuning_cache(str(p), True)
    text = p.read_text()
    assert text.startswith('{"bc_tuning": [')
    p.write_text('{"bc_tuning": [\n  {"log2_n": 12, "log2_avg_degree": 3, "log2_skew": 6, "batch_width": 64, '
                 '"alpha": 14.000, "group_vertices": 16, "rate": 1.0e+10}\n]}\n')
    bc.tuning_cache(str(p), False)
    q = tmp_path / "tune2.json"
    bc.tuning_cache(str(q), True)
    assert '"batch_width": 64' in q.read_text() and '"group_vertices": 16' in q.read_text()


def test_team_rule_without_gpu():
    # the team split of a traversal is host arithmetic; these are the splits the
    # measured calls ran (R-MAT 22: 128,304,910 arcs; R-MAT 12: about 6e4; a
    # grid of 444 blocks, 3 per SM)
    import paper_2305_03317_b300 as bc
    m22, m12, blocks, free = 128304910, 60000, 444, 270 * 10**9
    # R-MAT 22, 32 batches of 128: one block per 2^19 arcs would be one team;
    # two batches in flight
    assert bc.team_rule(m22, 128, 32, blocks, 5 * 10**9, free) == (2, 222)
    # one-source batches: teams of at most about 32 blocks, then the fewest
    # teams that need the same 20 rounds
    assert bc.team_rule(m22, 1, 256, blocks, 2 * 10**8, free) == (13, 34)
    # R-MAT 12: one block per one-source batch (4096 batches: 10 rounds of 410);
    # 128-wide batches on teams of about 0.7 m^0.24 blocks, no more teams than batches
    assert bc.team_rule(m12, 1, 4096, blocks, 10**6, free) == (410, 1)
    assert bc.team_rule(m12, 128, 32, blocks, 10**7, free) == (32, 13)
    # the slices within 30% of free memory and 24 GB
    assert bc.team_rule(m22, 1, 256, blocks, 10 * 10**9, free) == (2, 222)
    assert bc.team_rule(m22, 128, 32, blocks, 5 * 10**9, 10 * 10**9) == (1, 444)
    # asked-for counts, capped by batches; nothing to run still gives one team
    assert bc.team_rule(m22, 128, 32, blocks, 10**9, free, teams=4) == (4, 111)
    assert bc.team_rule(m12, 128, 32, blocks, 10**6, free, teams=100) == (32, 13)
    assert bc.team_rule(m12, 128, 0, blocks, 10**6, free) == (1, 444)
    with pytest.raises(bc.BCError) as ei:
        bc.team_rule(m12, 0, 32, blocks, 10**6, free)
    assert ei.value.status == bc.BC_E_INVALID_ARG
