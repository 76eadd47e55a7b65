"""The benchmark's byte accounting (host logic, no GPU): the algorithmic bytes behind
`roofline.achieved` are the per-unit figures of the Wilson roofline, and the ncu traffic ratio
behind `roofline.traffic` divides by the same formula for the kernel it was captured on."""
import bench


def test_roofline_units_per_site_and_link():
    """Spinor bytes per site, algorithmic link bytes per link, solution-increment bytes per site:
    FP64 24 reals (192 B) and 18-real links; FP32 and FP16 / BF16 12-real links, the half
    spinors with a 4-byte norm per site."""
    assert bench.spinor_link_bytes("fp64") == (192, 144, 192)
    assert bench.spinor_link_bytes("fp32") == (96, 48, 96)
    assert bench.spinor_link_bytes("fp16") == (52, 24, 52)
    assert bench.spinor_link_bytes("bf16") == (52, 24, 52)


def test_even_site_stencil_bytes_match_the_ncu_denominator():
    """One k_eo_even launch reads a spinor and writes one per odd-site half of every active slot,
    plus the links once: for the 32^3x16 capture with 12 slots that is the denominator the traffic
    entry stores, so the ratio it applies to the headline launch is traffic per algorithmic byte."""
    V = 32 * 32 * 32 * 16
    per_launch = bench.kernel_bytes("k_eo_even", "fp16", V, {"eo": 1, "rhs_iters": 12, "launches": 2}) / 2
    assert per_launch == (V // 2) * 2 * 52 * 12 + 4 * V * 24
    for entry in bench.NCU_TRAFFIC.values():
        assert entry["alg_bytes_all_slots"] == per_launch
        assert 1.0 <= entry["bytes_all_slots"] / entry["alg_bytes_all_slots"] < 1.5


def test_headline_even_site_launch_bytes():
    """At 32^3x64 with all 24 slots active one k_eo_even launch moves 2.818 GB algorithmic."""
    V = 32 * 32 * 32 * 64
    b = bench.kernel_bytes("k_eo_even", "fp16", V, {"eo": 1, "rhs_iters": 24, "launches": 2}) / 2
    assert b == (V // 2) * 104 * 24 + 4 * V * 24
    assert abs(b / 1e9 - 2.818) < 1e-3


def test_traffic_entry_is_keyed_to_the_kernel_source():
    """The traffic entry carries the hash of the sources it was captured on; a kernel whose hash
    differs finds no entry (the bench then reports traffic null)."""
    keys = list(bench.NCU_TRAFFIC)
    assert all(len(h) == 12 for _, h in keys)
    assert bench.NCU_TRAFFIC.get(("k_eo_even", "0" * 12)) is None
    h = bench.source_hash("k_eo_even")
    assert len(h) == 12 and h == bench.source_hash("k_eo_even")
