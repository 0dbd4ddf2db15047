"""The benchmark's roofline arithmetic, without a GPU: counted work turns into
flops with the per-primitive costs of the kernel table (six signed distances
of a prism's points to one plane 36 flop, a piece's four distances 24, an edge
intersection 10, a tetrahedron volume 17, a closed-form cut fraction 30, a
plane shift into the face frame 6; a positioning fill evaluation 30; a cubic's
coefficients from one swept triangle 110, one cubic evaluation 20), and the
phase flux's DRAM traffic is reported only while the kernel sources are the
captured ones."""
import hashlib
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORK = {"prism_planes": 1000.0, "piece_tests": 200.0, "edges": 300.0, "tet_volumes": 40.0,
        "cut_fractions": 10.0, "plane_shifts": 500.0, "faces": 7.0, "fill64": 11.0, "fill32": 13.0,
        "cubic_triangles": 3.0, "cubic_evals": 5.0, "reserved": 0.0}


def test_counted_flops_follow_the_unit_costs():
    import bench
    pf = 1000 * 36 + 200 * 24 + 300 * 10 + 40 * 17 + 10 * 30 + 500 * 6
    fixed64 = 11 * 30 + 3 * 110 + 5 * 20
    f32, f64, p = bench.work_flops(WORK, False)  # mixed form: the phase flux in FP32
    assert p == pf
    assert f32 == pf + 13 * 30
    assert f64 == fixed64
    f32, f64, p = bench.work_flops(WORK, True)   # plain form: the phase flux in FP64
    assert p == pf
    assert f32 == 13 * 30
    assert f64 == fixed64 + pf
    # faces and the reserved slot carry no flops
    w = dict(WORK, faces=1e9, reserved=1e9)
    assert bench.work_flops(w, False) == bench.work_flops(WORK, False)


def test_traffic_is_null_once_the_kernel_sources_change(monkeypatch):
    import bench
    key = ("deform3d", 128, "mixed")
    assert bench.captured_traffic(*key) in (None, bench.TRAFFIC[key]["bytes"])
    monkeypatch.setitem(bench.TRAFFIC, key, {"bytes": 1.0, "sources_sha256": "0" * 64})
    assert bench.captured_traffic(*key) is None
    h = hashlib.sha256()
    for f in bench.TRAFFIC_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    monkeypatch.setitem(bench.TRAFFIC, key, {"bytes": 2.0, "sources_sha256": h.hexdigest()})
    assert bench.captured_traffic(*key) == 2.0
    # no capture for other sizes or forms
    assert bench.captured_traffic("deform3d", 64, "mixed") is None
    assert bench.captured_traffic("deform3d", 128, "fp64") is None
