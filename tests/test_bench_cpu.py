"""CPU checks of bench.py's host logic: the algorithmic byte model of the
matvec passes, the whole-matvec roofline, and the rule that ncu traffic is
reported only while the kernel sources match the capture."""
import hashlib
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

# 96x64x32 ellipsoid: 102984 sites, padded 192 x 128 x 64
ELLIPSOID = {"Lx": 192, "Ly": 128, "Lz": 64, "ndipoles": 102984}


def test_pass_bytes_of_the_ellipsoid_at_32_rhs():
    """The per-launch algorithmic bytes quoted for the ellipsoid captures
    (x-fwd 381.9, y 906.0, z 1217.9, x-inv 461.1 MB at 32 RHS) follow from the
    model: compact vectors 3N s, padded intermediates 6Ms / 12Ms per RHS,
    index maps 4M (+N), the Green octant once."""
    mb = {k: bench.pass_bytes(k, ELLIPSOID, 32) / 1e6 for k in ("x_fwd_c64", "y_fwd_c64", "z_conv_c64", "x_inv_c64")}
    assert mb["x_fwd_c64"] == pytest.approx(381.9, abs=0.1)
    assert mb["y_fwd_c64"] == pytest.approx(906.0, abs=0.1)
    assert mb["z_conv_c64"] == pytest.approx(1217.9, abs=0.1)
    assert mb["x_inv_c64"] == pytest.approx(461.1, abs=0.1)
    assert bench.pass_bytes("y_inv_c64", ELLIPSOID, 32) == bench.pass_bytes("y_fwd_c64", ELLIPSOID, 32)
    assert bench.pass_bytes("z_conv_c128", ELLIPSOID, 32) == 2 * bench.pass_bytes("z_conv_c64", ELLIPSOID, 32)
    assert bench.pass_bytes("k_update_xr", ELLIPSOID, 32) is None


def _stats(ms, launches=10, units=320.0):
    return {"launches": launches, "ms": ms, "units": units}


def test_matvec_roofline_sums_the_passes():
    ks = {k: _stats(1.0) for k in ("x_fwd_c64", "y_fwd_c64", "z_conv_c64", "y_inv_c64", "x_inv_c64")}
    ks["bicgstab_c64"] = _stats(5.0)
    out = bench.matvec_roofline(ks, ELLIPSOID)
    want = sum(bench.pass_bytes(k, ELLIPSOID, 32) * 10 for k in ks if k != "bicgstab_c64")
    assert out["algorithmic_bytes"] == pytest.approx(want)
    assert out["achieved"] == pytest.approx(want / 5e-3 / 1e9)
    # counting only the RHS-matvecs a solve did (converged RHS skip their work)
    part = bench.matvec_roofline(ks, ELLIPSOID, rhs_matvecs=160)
    assert part["algorithmic_bytes"] < out["algorithmic_bytes"]
    del ks["y_inv_c64"]
    assert bench.matvec_roofline(ks, ELLIPSOID) is None     # neither 3 nor 5 passes


def test_captured_traffic_needs_matching_sources(tmp_path, monkeypatch):
    h = hashlib.sha256()
    for f in bench.KERNEL_SOURCES:
        h.update(open(os.path.join(ROOT, f), "rb").read())
    cur = h.hexdigest()[:16]
    for sha, want in ((cur, 12345), ("0" * 16, None)):
        md = tmp_path / f"cap_{sha}.md"
        md.write_text(f"source_sha256: {sha}\n\n### k_test<float> (1 us)\ntraffic_bytes_per_launch: 12345\n")
        monkeypatch.setattr(bench, "ROOT", ROOT)
        monkeypatch.setitem(bench.CAPTURES, ("x_fwd_c64", "wl", 4), (str(md), "k_test<float>"))
        assert bench.captured_traffic("x_fwd_c64", "wl", 4.0) == want
    assert bench.captured_traffic("x_fwd_c64", "other", 4.0) is None


def test_fused_update_traffic_is_counted_per_rhs_matvec():
    """Inside a solve the x passes also move the BiCGstab vectors: 5.5 compact
    vectors (3N complex each) per RHS-matvec on average."""
    ks = {k: _stats(1.0) for k in ("x_fwd_c64", "y_fwd_c64", "z_conv_c64", "y_inv_c64", "x_inv_c64")}
    plain = bench.matvec_roofline(ks, ELLIPSOID, rhs_matvecs=160)
    fused = bench.matvec_roofline(ks, ELLIPSOID, rhs_matvecs=160,
                                  fused_vectors=bench.FUSED_VECTORS_PER_MATVEC["bicgstab"])
    extra = 5.5 * 3 * ELLIPSOID["ndipoles"] * 8 * 160
    assert fused["fused_update_bytes"] == pytest.approx(extra)
    assert fused["algorithmic_bytes"] - plain["algorithmic_bytes"] == pytest.approx(extra)
