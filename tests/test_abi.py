"""CPU checks of the C ABI: the library builds for sm_103a, loads, and exports
every entry point that include/dgx.h declares (no GPU call is made)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(dgx_[a-z0-9_]+)\s*\(", src))
    return names


def test_library_exports_every_declared_symbol():
    from paper_2505_00384_gb300 import build, dgx
    path = build.build()
    lib = ctypes.CDLL(path)
    names = _declared()
    assert len(names) >= 15
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing
    bound = {s[0] for s in dgx.SIGNATURES}
    assert names <= bound, sorted(names - bound)


def test_binding_signatures_load():
    from paper_2505_00384_gb300 import dgx
    lib = dgx.load()
    assert lib.dgx_last_error(None) == b"null context"
    assert lib.dgx_num_dofs(None) == -1


def test_structs_match_header_layout():
    from paper_2505_00384_gb300 import dgx
    # 8 ints, 7 doubles, the 6-int refinement box; 2 ints then 7 doubles; mixed int/double padding
    assert ctypes.sizeof(dgx.dgx_mesh_desc) == 8 * 4 + 7 * 8 + 6 * 4
    assert ctypes.sizeof(dgx.dgx_background) == 2 * 4 + 7 * 8
    assert ctypes.sizeof(dgx.dgx_solve_opts) == 4 * 4 + 8 + 2 * 4 + 8 + 2 * 4
    assert ctypes.sizeof(dgx.dgx_solve_info) == 6 * 4 + 2 * 8
    # 2 ints, 5 doubles, one 64-bit seed, 2 ints; 4 ints then 5 doubles
    assert ctypes.sizeof(dgx.dgx_train_opts) == 2 * 4 + 5 * 8 + 8 + 2 * 4
    assert ctypes.sizeof(dgx.dgx_train_info) == 4 * 4 + 5 * 8
