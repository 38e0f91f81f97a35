"""The C-ABI library builds here, loads without a GPU and exports every function that
include/*.h declares (no compute calls: there is no GPU on this side)."""
import ctypes
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions(header="sf.h"):
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", header)):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \t\*]*?\b(sfc?_\w+)\s*\(", text, flags=re.M):
            line = text[m.start():text.find("\n", m.start())]
            if line.lstrip().startswith(("typedef", "#")):
                continue
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib_path():
    from paper_1701_04148_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = _declared_functions()
    for must in ("sf_create", "sf_insert_batch", "sf_delete_batch", "sf_export_slim", "sf_query_batch",
                 "sf_required_bytes", "sf_sync", "sf_destroy", "sf_update_batch"):
        assert must in names


def _exported(path):
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    return {ln.split()[-1] for ln in out.splitlines() if ln.strip()}


def test_library_exports_every_declared_symbol(lib_path):
    from paper_1701_04148_gb300 import build
    for path, header in ((lib_path, "sf.h"), (build.BENCH_LIB, "sf_bench.h")):
        L = ctypes.CDLL(path)
        missing = [n for n in sorted(_declared_functions(header)) if not hasattr(L, n)]
        assert not missing, f"declared in include/{header} but not exported by {os.path.basename(path)}: {missing}"
        assert _declared_functions(header) <= _exported(path)
    # the measurement kernels live only in the measurement library
    assert not (_declared_functions("sf_bench.h") & _exported(lib_path))


def test_binding_covers_the_header(lib_path):
    import paper_1701_04148_gb300 as sf
    assert _declared_functions("sf.h") <= set(sf.exported_symbols())
    assert _declared_functions("sf_bench.h") <= set(sf.exported_bench_symbols())


def test_argument_checks_need_no_gpu(lib_path):
    import paper_1701_04148_gb300 as sf
    L = sf.load(lib_path)
    assert L.sf_status_str(sf.SF_ERR_UNDERFLOW).decode().startswith("delete")
    bad = sf.make_params(0, 16, 16, 4, 1, 64)           # d = 0
    fb = ctypes.c_uint64()
    assert L.sf_required_bytes(ctypes.byref(bad), ctypes.byref(fb), None, None) == sf.SF_ERR_INVALID
    good = sf.make_params(4, 1 << 18, 16, 13, 2, 65536)
    fb, sb, xb = sf.required_bytes(good)
    assert fb == 4 * (1 << 18) * 16 * 4 and sb == 4 * (1 << 18) * 4
    assert xb >= 256 + 16 * 65536 * 32
    h = ctypes.c_void_p()
    assert L.sf_create(ctypes.byref(good), None, None, None, None, ctypes.byref(h)) == sf.SF_ERR_INVALID
    assert L.sf_insert_batch(None, None, 5) == sf.SF_ERR_INVALID
    assert L.sf_sync(None) == sf.SF_ERR_INVALID
    v = sf.SlimView(0, sf.SlimHeader(0, 1, 4, 16, 4, 1, 0), 0, 0)
    assert L.sf_query_batch(ctypes.byref(v), None, 0, None, None) == sf.SF_ERR_VERSION


def test_oracle_and_cuda_sources_share_nothing():
    """The oracle (test infrastructure) and the CUDA library include and import nothing of each other."""
    osrc = open(os.path.join(ROOT, "oracle", "sf_oracle.c")).read() + open(os.path.join(ROOT, "oracle", "__init__.py")).read()
    assert "paper_1701_04148_gb300" not in osrc and "csrc" not in osrc
    for p in glob.glob(os.path.join(ROOT, "paper_1701_04148_gb300", "**", "*.*"), recursive=True):
        if p.endswith((".cu", ".cuh", ".h", ".py")):
            txt = open(p).read()
            assert "import oracle" not in txt and "from oracle" not in txt and "sf_oracle" not in txt, p


def test_one_at_a_time_workspace_only_where_the_graph_path_applies(lib_path):
    """Chunk-1 sketches reserve the dependency-graph workspace when they are at least 1,024 wide
    and w * z stays below 2^32 (the per-counter sort key has a spare value); others use the
    window kernel and need only the control words."""
    import paper_1701_04148_gb300 as sf
    sf.load(lib_path)
    _, _, graph = sf.required_bytes(sf.make_params(4, 4096, 16, 4, 1, 1))
    _, _, narrow = sf.required_bytes(sf.make_params(4, 1000, 16, 4, 1, 1))
    _, _, wide = sf.required_bytes(sf.make_params(1, 1 << 28, 16, 4, 1, 1))       # w * z = 2^32
    _, _, just_under = sf.required_bytes(sf.make_params(1, (1 << 28) - 1, 16, 4, 1, 1))
    assert narrow < 4096 and wide < 4096
    assert graph > 30_000_000 and just_under > 10_000_000


def test_shared_dictionary_sizes(lib_path):
    """Host-only arithmetic of the boundary: a sketch created with SF_FLAG_SHARED_DICT needs no
    dictionary in its scratch, and sf_dictionary_bytes gives the one it then takes from elsewhere
    (32 B x a power of two >= 16 S slots up to S = 65,536, >= 8 S above; none for S = 1)."""
    import paper_1701_04148_gb300 as sf
    L = sf.load(lib_path)

    def sizes(chunk, flags):
        p = sf.make_params(4, 4096, 16, 4, 1, chunk, flags)
        fb, sb, xb, db = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
        assert L.sf_required_bytes(ctypes.byref(p), ctypes.byref(fb), ctypes.byref(sb), ctypes.byref(xb)) == 0
        assert L.sf_dictionary_bytes(ctypes.byref(p), ctypes.byref(db)) == 0
        return xb.value, db.value

    for chunk, slots in ((1000, 16384), (65536, 1 << 20), (65537, 1 << 20), (100000, 1 << 20), (1 << 20, 1 << 23)):
        own, d_own = sizes(chunk, 0)
        shared, d_shared = sizes(chunk, sf.SF_FLAG_SHARED_DICT)
        assert d_own == d_shared == 32 * slots, chunk
        assert own - shared == 32 * slots, chunk
    assert sizes(1, sf.SF_FLAG_SHARED_DICT)[1] == 0
