"""The C-ABI library builds, loads and exports every entry point that
include/sph.h declares (no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "sph.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?(?:int|void|char)\s*\*?\s*(sph_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def built_lib():
    from paper_2510_25702_gb300 import build

    return build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("sph_create", "sph_add_buffer", "sph_step", "sph_read_fields", "sph_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(built_lib):
    lib = ctypes.CDLL(built_lib)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_header(built_lib):
    from paper_2510_25702_gb300 import sph

    assert set(sph.EXPORTS) == set(declared_functions())


def test_error_strings_without_gpu(built_lib):
    from paper_2510_25702_gb300 import sph

    L = sph.lib()
    assert L.sph_abi_version() == 3
    for code, name in sph.ERRORS.items():
        assert L.sph_error_string(code)
    assert L.sph_error_string(0) == b"ok"


def test_struct_sizes_match_header(built_lib):
    """ctypes mirrors have the C layout: compile a probe that prints sizeof."""
    import subprocess
    import tempfile

    from paper_2510_25702_gb300 import sph

    probe = r'''
#include <stdio.h>
#include <stddef.h>
#include "sph.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\n", sizeof(sph_config), sizeof(sph_particles),
         sizeof(sph_buffer_desc), sizeof(sph_alloc), sizeof(sph_stats), offsetof(sph_config, dp),
         offsetof(sph_buffer_desc, theta), offsetof(sph_config, obc), offsetof(sph_config, density_sum),
         offsetof(sph_config, tvf_alpha), offsetof(sph_config, wall_function), offsetof(sph_config, tvf_pbuf));
  return 0;
}
'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "p.c")
        open(c, "w").write(probe)
        exe = os.path.join(d, "p")
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe])
        out = [int(x) for x in subprocess.check_output([exe]).split()]
    expect = [ctypes.sizeof(sph.Config), ctypes.sizeof(sph.Particles), ctypes.sizeof(sph.BufferDesc),
              ctypes.sizeof(sph.Alloc), ctypes.sizeof(sph.Stats), sph.Config.dp.offset,
              sph.BufferDesc.theta.offset, sph.Config.obc.offset, sph.Config.density_sum.offset,
              sph.Config.tvf_alpha.offset, sph.Config.wall_function.offset, sph.Config.tvf_pbuf.offset]
    assert out == expect


def test_oracle_struct_layout_matches_its_header():
    """The oracle's ctypes mirrors have its C layout (the switches at the
    end of orc_config included)."""
    import subprocess
    import tempfile

    import oracle

    probe = r'''
#include <stdio.h>
#include <stddef.h>
#include "sph_oracle.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu\n", sizeof(orc_config), sizeof(orc_buffer), sizeof(orc_state),
         offsetof(orc_config, density_sum), offsetof(orc_config, wall_fn), offsetof(orc_config, tvf_pbuf),
         offsetof(orc_config, tvf_alpha));
  return 0;
}
'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "p.c")
        open(c, "w").write(probe)
        exe = os.path.join(d, "p")
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "oracle"), c, "-o", exe])
        out = [int(x) for x in subprocess.check_output([exe]).split()]
    C = oracle.OrcConfig
    expect = [ctypes.sizeof(C), ctypes.sizeof(oracle.OrcBuffer), ctypes.sizeof(oracle.OrcState),
              C.density_sum.offset, C.wall_fn.offset, C.tvf_pbuf.offset, C.tvf_alpha.offset]
    assert out == expect
