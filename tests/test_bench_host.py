"""Host-side pieces of bench.py that set the numbers its JSON line reports:
the FP32 ceiling of the gather, the counted arithmetic per cell-velocity,
and the DRAM traffic taken from the committed ncu summary only while the
gather's sources and tiling are those the counters were taken on.  No GPU.
"""
import hashlib
import os
import types

import pytest

import bench


class _FakeTorch:
    """The two device queries _fp32_peak makes, answered as a GB300 would."""
    class cuda:
        @staticmethod
        def current_device():
            return 0

        @staticmethod
        def get_device_properties(i):
            return types.SimpleNamespace(multi_processor_count=152)


def test_fp32_peak_from_unit_counts_and_clock():
    # 152 SMs x 128 FP32 lanes x 2 flops per FMA x 2070 MHz, both read from the device
    peak, n_sm, mhz = bench._fp32_peak(_FakeTorch, 2070.0)
    assert (n_sm, mhz) == (152, 2070.0)
    assert peak == pytest.approx(80.54784, rel=1e-12)
    half, _, _ = bench._fp32_peak(_FakeTorch, 1035.0)
    assert half == pytest.approx(peak / 2, rel=1e-12)


@pytest.mark.parametrize("D,NC,nf,flops", [(2, 2, 3, 407), (3, 1, 4, 402)])
def test_counted_gather_arithmetic(D, NC, nf, flops):
    """The per-cell-velocity counts stated with the benchmark: triangles
    132 (slope) + 3 x 77 (faces) + 44 (stage 1); tetrahedra 104 + 4 x 64 + 42."""
    assert bench._gather_flops_per_cvu(D, NC, nf) == flops


def test_counted_arithmetic_grows_with_faces_per_cell():
    """A quadrilateral (four faces) costs one more face flux and four more
    limiter evaluations than a triangle."""
    tri, quad = bench._gather_flops_per_cvu(2, 2, 3), bench._gather_flops_per_cvu(2, 2, 4)
    assert quad - tri == 77 + 2 * ((1 + 4) + (4 + 10))


def _profile_fields(workload):
    prof = os.path.join(bench.ROOT, "profiles", bench.TRAFFIC_PROFILES[workload])
    out = {}
    for line in open(prof):
        if ":" in line and line.split(":")[0] in ("gather-sources-sha256-16", "traffic-bytes-per-launch",
                                                  "traffic-tiling"):
            k, v = line.split(":", 1)
            out[k] = v.strip()
    return out


@pytest.mark.parametrize("workload", sorted(bench.TRAFFIC_PROFILES))
def test_traffic_is_reported_only_for_the_profiled_kernel_and_tiling(workload):
    if not os.path.exists(os.path.join(bench.ROOT, "profiles", bench.TRAFFIC_PROFILES[workload])):
        pytest.skip("no committed traffic summary for this workload")
    fields = _profile_fields(workload)
    h = hashlib.sha256()
    h.update(bench._gather_sources())
    tiling = dict(kv.split(" ") for kv in fields["traffic-tiling"].split(", "))
    args = (int(tiling["patch"]), int(tiling["vtile"]), int(tiling["threads"]), int(tiling["group"]))
    got = bench._gather_traffic(workload, *args)
    if fields["gather-sources-sha256-16"] == h.hexdigest()[:16]:
        assert got == int(fields["traffic-bytes-per-launch"])
    else:
        assert got is None
    # another tiling, or another workload, never borrows the figure
    assert bench._gather_traffic(workload, args[0], args[1], args[2], args[3] + 1) is None
    assert bench._gather_traffic(workload, args[0] + 1, *args[1:]) is None
    assert bench._gather_traffic("sphere_Ma4_Kn0.1_tet150k_v28", *args) is None
