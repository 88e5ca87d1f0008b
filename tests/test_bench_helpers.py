"""The bench's host-side arithmetic (no GPU): the algorithmic bytes and flops
of one H per 5D site, and the roofline and flop-rate figures computed from a
hop profile."""
import bench
import synthetic as sy


def _w(c):
    return sy.WORKLOADS["cfg5_32x32x32x64_ls16_mobius_3lvl" if c else "cfg2_16x16x16x16_ls16_shamir"]


def test_operator_bytes_per_site():
    # (240 + 576 / Ls) reals: 4 passes x (24 in + 24 out), 2 x 24 self terms,
    # 8 links of 18 reals per 4D site shared by the Ls slices, in each pass
    for w in (_w(True), _w(False)):
        reals = 4 * (24 + 24) + 2 * 24 + 4 * 8 * 18 / w.Ls
        assert bench.operator_bytes_per_site(w, 2) == 2 * reals
    assert bench.operator_bytes_per_site(_w(True), 2) == 552.0


def test_hop_flops_per_site():
    # Ls 16: Shamir 6528, Moebius 7248 (the Moebius K on the eight neighbours
    # of pass A and the K of passes A, C and D: 8 x 72 + 3 x (72 - 24) more)
    assert bench.hop_flops_per_site(_w(False)) == 6528
    assert bench.hop_flops_per_site(_w(True)) == 7248
    assert bench.hop_flops_per_site(_w(True)) - bench.hop_flops_per_site(_w(False)) == 8 * 72 + 3 * (72 - 24)


def test_roofline_and_flop_rate_from_a_profile():
    w = _w(True)
    n5 = bench.n5_of(w)
    ms, launches = 1000.0, 400
    op = launches * n5 * bench.operator_bytes_per_site(w, 2) / 4
    hop_all = {"f16": {"launches": launches, "ms": ms, "bytes": 1.5 * op, "op_bytes": op}}
    r = bench.roofline(w, hop_all, "f16", 6658.0, "measured", 1)
    assert abs(r["achieved"] - 1.5 * op / 1.0 / 1e9) < 1e-6 * r["achieved"]
    assert abs(r["achieved_operator_bytes_only"] - op / 1e9) < 1e-6 * r["achieved"]
    assert abs(r["frac"] - r["achieved"] / 6658.0) < 1e-12
    assert r["avg_launch_us"] == ms * 1e3 / launches
    assert r["traffic"] == bench.HOP_TRAFFIC[w.name]
    f = bench.hop_flop_rate(w, hop_all, "f16")
    assert abs(f["achieved"] - launches / 4 * n5 * 7248 / 1.0 / 1e12) < 1e-9
    assert bench.roofline(w, hop_all, "f32", 6658.0, "measured", 1) is None
    assert bench.hop_flop_rate(w, hop_all, "f32") is None
