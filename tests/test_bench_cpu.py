"""Host-side checks of bench.py that need no GPU: the kernel-launch count it claims per matvec
(`gpu_launches`) against the launch lists that ncu recorded for the same configurations
(profiles/launches_*.md, one metric pass over the timed steps), and the roofline arithmetic of the
GMRES overhead."""
import os
import re

import pytest

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def launches_in_summary(name):
    """Kernel launches per matvec in a launch-list summary (the per-kernel table; the L2 flush
    row, a torch fill between steps, is not one of the library's kernels)."""
    text = open(os.path.join(ROOT, "profiles", name)).read()
    total = 0
    for m in re.finditer(r"^\| `([^`]+)` \| (\d+) \|", text, flags=re.M):
        if not m.group(1).startswith("L2 flush"):
            total += int(m.group(2))
    return total


@pytest.mark.parametrize("summary,precision,nr,p,rotation", [
    ("launches_silver_sphere_s7_fp64_p10.md", "fp64", 1, 10, True),
    ("launches_silver_sphere_s7_fp32_p10.md", "fp32", 1, 10, True),
    ("launches_silver_sphere_s7_bf16x3_p10.md", "bf16x3", 1, 10, True),
    ("launches_torus_512x128_bf16x3_128rhs.md", "bf16x3", 128, 8, False),
])
def test_launch_count_matches_the_ncu_launch_lists(summary, precision, nr, p, rotation):
    # l_max = 5 on both meshes at these leaf sizes; two multipole domains
    assert bench.launches_per_matvec(5, nr, 2, precision, p, rotation) == launches_in_summary(summary)


def test_gmres_roofline_counts_products_without_the_first_residual():
    # x0 = 0: one cycle of 50 steps makes 50 Arnoldi products and one final true residual
    r = bench.gmres_roofline(1000, 50, 50, ms_total=51 * 2.0 + 50 * 0.5, matvec_ms=2.0)
    assert r["products"] == 51
    assert abs(r["ms_per_step"] - 0.5) < 1e-12
