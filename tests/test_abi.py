"""CPU checks of the C ABI: the library loads without a GPU, exports every
function include/bf.h declares, and rejects bad arguments before touching a
device.  No compute call runs here."""
import ctypes as C
import os
import re

import pytest

from paper_1802_01685_gb300 import bf
from paper_1802_01685_gb300 import build as bfbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "bf.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(bf_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    bfbuild.build()
    return bf.load()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 25
    raw = C.CDLL(bf.LIB_PATH)
    missing = [n for n in names if not hasattr(raw, n)]
    assert not missing, missing


def test_binding_covers_the_header(lib):
    src = open(bf.__file__).read()
    for n in declared_functions():
        assert f'"{n}"' in src, n


def test_status_strings_and_version(lib):
    assert bf.bf_abi_version() == 2
    assert bf.bf_status_string(bf.BF_OK) == "ok"
    assert bf.bf_status_string(bf.BF_EINVAL) == "invalid argument"
    assert bf.bf_status_string(99) == "unknown status"


def test_defaults(lib):
    c = bf.bf_config_default()
    assert c.max_candidates == 1 << 22 and c.serve_slots == 8 and c.serve_queue == 1024
    assert c.serve_policy == bf.BF_SERVE_FAIR
    o = bf.bf_opts_default()
    assert o.precision == bf.BF_SPLIT_BF16 and o.kappa == 5.0 and o.hist_bins == 1024
    assert abs(o.map_dt_s - 1e-3) < 1e-15 and o.map_df_hz == 4.0 and o.rho_out is None


def test_null_arguments_are_rejected(lib):
    assert lib.bf_init(None, None) == bf.BF_EINVAL
    h = C.c_void_p()
    assert lib.bf_bank_create(None, None, 0, 2048.0, 1.0, 3, C.byref(h)) == bf.BF_EINVAL
    assert lib.bf_correlate(None, None, None, None, 0, 2048.0, None, C.byref(h)) == bf.BF_EINVAL
    assert lib.bf_control_randomize(None, None, 10, 1, None) == bf.BF_EINVAL
    assert lib.bf_serve_submit(None, None, None) == bf.BF_EINVAL
    assert lib.bf_result_info_get(None, None) == bf.BF_EINVAL
    assert lib.bf_result_copy_to_host(None, 0, None, None, None, None, None) == bf.BF_EINVAL
    assert lib.bf_result_copy_to_host_async(None, 0, None, None, None, None, None, None) == bf.BF_EINVAL
    assert "NULL" in bf.bf_last_error() or bf.bf_last_error()
    lib.bf_destroy(None)
    lib.bf_result_destroy(None)
    lib.bf_bank_destroy(None)


def test_init_without_gpu_fails_cleanly(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = C.c_void_p()
    st = lib.bf_init(None, C.byref(h))
    assert st in (bf.BF_ECUDA, bf.BF_EINVAL, bf.BF_ENOTSUP)
    assert h.value is None
    assert bf.bf_last_error()


def test_struct_layouts_match_the_header(lib, tmp_path):
    """Compiles a probe against include/bf.h and compares every field offset and
    struct size with the ctypes mirror."""
    structs = {"bf_config": bf.bf_config, "bf_chirp": bf.bf_chirp,
               "bf_chirp_grid": bf.bf_chirp_grid, "bf_opts": bf.bf_opts,
               "bf_result_info": bf.bf_result_info, "bf_request": bf.bf_request,
               "bf_serve_stats": bf.bf_serve_stats, "bf_tail": bf.bf_tail,
               "bf_skewnorm": bf.bf_skewnorm}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "bf.h"', "int main(void){"]
    for name, cls in structs.items():
        lines.append(f'printf("{name} size %zu\\n", sizeof({name}));')
        for fname, _ in cls._fields_:
            lines.append(f'printf("{name} {fname} %zu\\n", offsetof({name}, {fname}));')
    lines.append("return 0;}")
    src = tmp_path / "probe.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "probe"
    import subprocess
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    for line in filter(None, out):
        name, field, val = line.split()
        cls = structs[name]
        if field == "size":
            assert C.sizeof(cls) == int(val), (name, C.sizeof(cls), val)
        else:
            assert getattr(cls, field).offset == int(val), (name, field)
