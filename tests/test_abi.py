"""CPU checks of the C-ABI library: it builds for sm_103a, loads, exports
every function include/atp.h declares, and the ctypes structs of the binding
have the C layout (checked against gcc's own sizeof/offsetof of the header).
No compute call is made here."""
import ctypes as C
import os
import re
import subprocess
import tempfile

import pytest

from paper_2603_20525_gb300 import atp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "atp.h")


def declared():
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:int|size_t|const char \*)\s*(atp_\w+)\s*\(", txt, re.M)))


def test_header_declarations_are_exported():
    names = declared()
    assert names == sorted(atp.EXPORTS)
    L = atp.load()
    for n in names:
        assert isinstance(getattr(L, n), C._CFuncPtr), n


def test_version_and_sizes_without_gpu():
    L = atp.load()
    ver = int(re.search(r"#define ATP_VERSION (\d+)", open(HEADER).read()).group(1))
    assert L.atp_version() == ver
    assert L.atp_terrain_bytes(1024, 1024, atp.F32X4) == 1024 * 1024 * 16
    assert L.atp_terrain_bytes(512, 256, atp.BF16X4) == 512 * 256 * 8 + 64 * 32 * 16
    assert L.atp_terrain_bytes(13, 9, atp.BF16X4) == 1024 + 2 * 2 * 16   # 936 B -> 1024
    assert L.atp_terrain_bytes(0, 5, atp.F32X4) == 0


def test_struct_layout_matches_header():
    src = r'''
#include <stdio.h>
#include <stddef.h>
#include "atp.h"
#define P(T) printf(#T " %zu\n", sizeof(T));
#define O(T, f) printf(#T "." #f " %zu\n", offsetof(T, f));
int main(void) {
  P(atp_vehicle) P(atp_cost) P(atp_state) P(atp_terrain) P(atp_plan_out)
  P(atp_est_state) P(atp_plan_request)
  O(atp_vehicle, g) O(atp_cost, goal_r) O(atp_state, delta) O(atp_terrain, format)
  O(atp_terrain, cell) O(atp_terrain, flags) O(atp_plan_out, best_min_step)
  O(atp_est_state, vx) O(atp_plan_request, cand_xf_dev) O(atp_plan_request, dt)
  return 0;
}
'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "l.c")
        open(c, "w").write(src)
        exe = os.path.join(d, "l")
        subprocess.run(["gcc", "-I", os.path.dirname(HEADER), c, "-o", exe], check=True)
        out = dict(l.rsplit(" ", 1) for l in subprocess.run([exe], capture_output=True,
                                                            text=True, check=True).stdout.split("\n") if l)
    assert int(out["atp_vehicle"]) == C.sizeof(atp.Vehicle)
    assert int(out["atp_cost"]) == C.sizeof(atp.Cost)
    assert int(out["atp_state"]) == C.sizeof(atp.State)
    assert int(out["atp_terrain"]) == C.sizeof(atp.TerrainC)
    assert int(out["atp_plan_out"]) == C.sizeof(atp.PlanOut) == 24
    assert int(out["atp_vehicle.g"]) == atp.Vehicle.g.offset
    assert int(out["atp_cost.goal_r"]) == atp.Cost.goal_r.offset
    assert int(out["atp_state.delta"]) == atp.State.delta.offset
    assert int(out["atp_terrain.format"]) == atp.TerrainC.format.offset
    assert int(out["atp_terrain.cell"]) == atp.TerrainC.cell.offset
    assert int(out["atp_plan_out.best_min_step"]) == atp.PlanOut.best_min_step.offset
    assert int(out["atp_terrain.flags"]) == atp.TerrainC.flags.offset
    assert int(out["atp_est_state"]) == C.sizeof(atp.EstState)
    assert int(out["atp_est_state.vx"]) == atp.EstState.vx.offset
    assert int(out["atp_plan_request"]) == C.sizeof(atp.PlanRequest)
    assert int(out["atp_plan_request.cand_xf_dev"]) == atp.PlanRequest.cand_xf_dev.offset
    assert int(out["atp_plan_request.dt"]) == atp.PlanRequest.dt.offset


def test_no_cpu_fallback_path():
    """The binding has no compute of its own: every planner entry point goes
    through the library, and the package never imports the oracle."""
    import paper_2603_20525_gb300 as pkg
    for root, _, files in os.walk(os.path.dirname(pkg.__file__)):
        for f in files:
            if f.endswith(".py"):
                txt = open(os.path.join(root, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f


def test_create_without_device_is_an_error_not_a_crash():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    L = atp.load()
    h = C.c_void_p()
    assert L.atp_create(C.byref(h), 0) != 0
    assert not h.value
