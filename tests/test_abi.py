"""The C-ABI library builds, loads without a GPU and exports every entry
point include/tg.h declares; the binding's structs match the header."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2606_22332_gb300 import build

    try:
        return build.build()
    except RuntimeError as e:  # no nvcc on this machine
        pytest.skip(str(e))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "tg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tg_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("tg_create_scene", "tg_upload_objects", "tg_step_sensors", "tg_read_taxels"):
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_lists_every_symbol(libpath):
    import paper_2606_22332_gb300.tg as tg

    assert sorted(tg.EXPORTED) == declared_functions()


def test_struct_sizes_match_header(libpath):
    """Compile a tiny C program against tg.h and compare sizeof/offsetof with ctypes."""
    import subprocess
    import tempfile

    import paper_2606_22332_gb300.tg as tg

    prog = r'''
#include <stdio.h>
#include <stddef.h>
#include "tg.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu\n", sizeof(tg_params), sizeof(tg_scene_desc), sizeof(tg_object_desc),
         sizeof(tg_step_inputs), sizeof(tg_noise_group));
  printf("%zu %zu %zu\n", offsetof(tg_scene_desc, params), offsetof(tg_scene_desc, sensors),
         offsetof(tg_object_desc, values));
  printf("%zu %zu %zu\n", sizeof(tg_tune_report), offsetof(tg_tune_report, cand), offsetof(tg_params, dr_scale));
  return 0; }
'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        open(c, "w").write(prog)
        exe = os.path.join(d, "t")
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()
    sizes = [int(v) for v in out]
    assert sizes[:5] == [ctypes.sizeof(tg.Params), ctypes.sizeof(tg.SceneDesc), ctypes.sizeof(tg.ObjectDesc),
                         ctypes.sizeof(tg.StepInputs), ctypes.sizeof(tg.NoiseGroup)]
    assert sizes[5:8] == [tg.SceneDesc.params.offset, tg.SceneDesc.sensors.offset, tg.ObjectDesc.values.offset]
    assert sizes[8:] == [ctypes.sizeof(tg.TuneReport), tg.TuneReport.cand.offset, tg.Params.dr_scale.offset]


def test_max_link_taxels(libpath):
    import paper_2606_22332_gb300.tg as tg

    assert tg.lib().tg_max_link_taxels() >= 1000


def test_binding_names_every_schedule(libpath):
    """tg.SCHEDULES names the header's tg_schedule values in order (the
    autotuner's report and tg_set_schedule index them)."""
    import paper_2606_22332_gb300.tg as tg

    src = open(os.path.join(ROOT, "include", "tg.h")).read()
    body = re.search(r"typedef enum \{([^}]*)\} tg_schedule;", src, flags=re.S).group(1)
    vals = dict((k, int(v)) for k, v in re.findall(r"(TG_SCHED_[A-Z_0-9]+)\s*=\s*(\d+)", body))
    assert vals["TG_SCHED_COUNT"] == len(tg.SCHEDULES)
    expect = {"grid": "TG_SCHED_GRID", "persistent": "TG_SCHED_PERSISTENT", "pipe1024": "TG_SCHED_PIPE_1024",
              "pipe768": "TG_SCHED_PIPE_768", "pipe512": "TG_SCHED_PIPE_512", "grid384": "TG_SCHED_GRID_384",
              "persistent384": "TG_SCHED_PERSISTENT_384"}
    for i, name in enumerate(tg.SCHEDULES):
        assert vals[expect[name]] == i, name


def test_create_scene_rejects_too_many_taxels_on_the_host(libpath):
    """A scene indexes its per-taxel arrays with 32 bits: tg_create_scene
    refuses 2^31 taxels or more before it touches the GPU."""
    import numpy as np

    import paper_2606_22332_gb300.tg as tg

    offs = np.array([0, 1 << 31], np.int64)
    rows = np.ones(1, np.int32)
    cols = np.ones(1, np.int32)
    d = tg.SceneDesc()
    d.n_envs, d.max_links = 1, 1
    d.taxel_offsets, d.link_rows, d.link_cols = offs.ctypes.data, rows.ctypes.data, cols.ctypes.data
    h = ctypes.c_void_p()
    st = tg.lib().tg_create_scene(ctypes.byref(d), ctypes.byref(h))
    assert st == 1 and not h.value  # TG_ERR_INVALID_ARG, no scene
    assert b"2^31" in tg.lib().tg_last_error(None)
