"""The C-ABI library loads and exports every function include/gbt.h declares
(no GPU needed: nothing here launches a kernel)."""
import ctypes
import os

import pytest

from paper_2501_13382_gb300 import gbt


def _built():
    return os.path.exists(gbt.LIB_PATH)


def test_header_declares_the_boundary():
    names = gbt.declared_functions()
    for n in ("gbt_scene_create", "gbt_trace", "gbt_sum", "gbt_sum_backward", "gbt_batch_submit",
              "gbt_solve", "gbt_sync", "gbt_last_error"):
        assert n in names


@pytest.fixture(scope="module")
def lib():
    if not _built():
        from paper_2501_13382_gb300 import build
        build.build()
    return gbt.load()


def test_library_exports_every_declared_symbol(lib):
    raw = ctypes.CDLL(gbt.LIB_PATH)
    for name in gbt.declared_functions():
        assert hasattr(raw, name), f"libgbt.so does not export {name}"
    assert set(gbt._SIGS) >= set(gbt.declared_functions())


def test_version_and_error_string_without_gpu(lib):
    assert gbt.gbt_version() == 2
    assert isinstance(lib.gbt_last_error(), bytes)


def test_launch_counter_reads_without_gpu(lib):
    gbt.gbt_launches_read(reset=True)
    assert gbt.gbt_launches_read(reset=False) == 0      # nothing launched on a host-only run


def test_struct_layouts_match_header_sizes(lib):
    # the C compiler's view of the argument structs, compiled here from the header
    import subprocess, tempfile
    src = r'''
#include <stdio.h>
#include <stddef.h>
#include "gbt.h"
int main(void){
 printf("%zu %zu %zu %zu %zu\n", sizeof(gbt_scene_desc), sizeof(gbt_source_desc),
        sizeof(gbt_trace_info), sizeof(gbt_sum_args), sizeof(gbt_batch_desc));
 printf("%zu %zu %zu\n", offsetof(gbt_sum_args, gamma), offsetof(gbt_sum_args, cutoff),
        offsetof(gbt_sum_args, max_device_bytes));
 printf("%zu %zu\n", offsetof(gbt_sum_args, absorption), offsetof(gbt_sum_args, flow_resistivity));
 return 0;}
'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c"); exe = os.path.join(d, "t")
        open(c, "w").write(src)
        subprocess.run(["gcc", "-I", os.path.dirname(gbt.HEADER_PATH), c, "-o", exe], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()
    sizes = [int(v) for v in out]
    assert sizes[:5] == [ctypes.sizeof(gbt.gbt_scene_desc), ctypes.sizeof(gbt.gbt_source_desc),
                         ctypes.sizeof(gbt.gbt_trace_info), ctypes.sizeof(gbt.gbt_sum_args),
                         ctypes.sizeof(gbt.gbt_batch_desc)]
    assert sizes[5:] == [gbt.gbt_sum_args.gamma.offset, gbt.gbt_sum_args.cutoff.offset,
                         gbt.gbt_sum_args.max_device_bytes.offset,
                         gbt.gbt_sum_args.absorption.offset,
                         gbt.gbt_sum_args.flow_resistivity.offset]


def test_library_air_absorption_equals_the_oracles(lib):
    """gbt_air_absorption (host code of the library, ISO 9613-1) against the oracle's
    independent implementation, itself pinned to the standard's table; no GPU involved."""
    import numpy as np
    from oracle import oracle as O
    f = np.geomspace(20.0, 20000.0, 31)
    for T, rh, p in ((20.0, 70.0, 101.325), (-10.0, 20.0, 90.0), (35.0, 95.0, 105.0),
                     (15.0, 0.0, 101.325)):
        mine = gbt.gbt_air_absorption(f, T, rh, p)
        ref = O.air_absorption(f, T, rh, p)
        assert np.allclose(mine, ref, rtol=1e-12, atol=0), (T, rh, p)
    with pytest.raises(gbt.GBTError):
        gbt.gbt_air_absorption([1000.0], 20.0, 120.0, 101.325)
    with pytest.raises(gbt.GBTError):
        gbt.gbt_air_absorption([-5.0], 20.0, 50.0, 101.325)


def test_list_capacity_setter_checks_its_argument(lib):
    """gbt_list_capacity_set is host state only: any entries >= 0 is taken (0 restores the
    default), a negative bound is rejected."""
    gbt.gbt_list_capacity_set(1 << 20)
    gbt.gbt_list_capacity_set(0)
    with pytest.raises(gbt.GBTError):
        gbt.gbt_list_capacity_set(-1)
