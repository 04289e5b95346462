"""The C-ABI library loads and exports every entry point include/tstar.h declares (no GPU needed)."""
import ctypes
import os

import pytest

from paper_2405_09233_gb300 import binding


def test_library_exports_every_declared_symbol():
    if not os.path.exists(binding.LIB_PATH):
        pytest.skip("libtstar.so not built")
    L = binding.lib()
    declared = binding.declared_symbols()
    assert len(declared) >= 12
    missing = [s for s in declared if not hasattr(L, s)]
    assert not missing, f"declared but not exported: {missing}"
    # every declared symbol is also bound by the Python wrapper
    assert set(declared) <= set(binding._SIGNATURES), set(declared) - set(binding._SIGNATURES)


def test_host_only_calls():
    """Calls that touch no device: status names and option defaults."""
    if not os.path.exists(binding.LIB_PATH):
        pytest.skip("libtstar.so not built")
    L = binding.lib()
    assert L.ts_status_string(0) == b"TS_OK"
    assert L.ts_status_string(-4) == b"TS_ERR_NONFINITE"
    o = binding.SolveOpts()
    L.ts_solve_opts_default(ctypes.byref(o))
    assert (o.restart, o.max_restarts, o.tol, o.precision) == (20, 200, 1e-10, 0)
    assert L.ts_last_error(None) == b"null context"


def test_struct_layouts_match_header():
    """The ctypes mirrors of ts_solve_opts / ts_solve_info / ts_stats / ts_instance have the header's
    field order."""
    import re
    text = open(os.path.join(os.path.dirname(binding.LIB_PATH), "..", "include", "tstar.h")).read()
    for cls, tag in ((binding.SolveOpts, "ts_solve_opts"), (binding.SolveInfo, "ts_solve_info"),
                     (binding.Stats, "ts_stats"), (binding.Instance, "ts_instance")):
        body = re.search(r"typedef struct \{([^{}]*)\}\s*" + tag + ";", text).group(1)
        body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
        names = []
        for decl in body.split(";"):
            decl = decl.strip()
            if not decl:
                continue
            chunks = decl.replace("*", " ").split(",")
            names.append(chunks[0].split()[-1])          # "long long launches" -> "launches"
            names += [c.strip() for c in chunks[1:]]
        assert [f[0] for f in cls._fields_] == [n.strip() for n in names if n.strip()], tag
