"""Host-side logic of bench.py (CPU only): the contract's defaults, the kernel labels and the
committed-traffic lookup, which must return a figure only for the kernel source and variant it
was measured on."""
import json
import os
import sys

import bench


def _parse(argv):
    old = sys.argv
    sys.argv = ["bench.py"] + argv
    try:
        return bench.parse()
    finally:
        sys.argv = old


def test_defaults_follow_the_timing_contract():
    a = _parse([])
    assert a.gpus == 1 and a.config == 5 and a.impl == "ours"   # the largest single-GPU configuration
    assert a.warmup >= 3 and a.steps >= 1
    assert a.snapshot == "bf16"                                  # the configuration's own
    assert _parse(["--config", "2"]).snapshot == "fp16"
    assert _parse(["--config", "5", "--snapshot", "fp32"]).snapshot == "fp32"


def test_kernel_labels_name_the_source_files():
    assert bench.kernel_label(3, False)[1] == "stencil2d_pipe.cu"
    assert bench.kernel_label(0, True)[1] == "stencil2d.cu"
    assert bench.kernel_label(0, False, ndim=3)[1] == "stencil3d.cu"
    assert "k_adj3d_cl<G=4" in bench.kernel_label(0, True, ndim=3, cluster=True, group=4)[0]
    assert bench.kernel_label(2, True, ndim=3)[0].startswith("k_step3d_ws<ADJ>")
    assert bench.kernel_label(3, True, ndim=3)[0].startswith("k_step3d_ws[last-warp refill]<ADJ>")
    assert bench.kernel_label(0, True, ndim=3)[0].startswith("k_step3d<ADJ>")
    assert bench.kernel_label(3, False, time_block=2)[0].startswith("k_fwd2d_tb")
    assert bench.kernel_label(3, False, time_block=1)[0].startswith("k_fwd2d_ws")   # one level per launch
    for args in ((3, False), (2, True), (0, False), (0, True)):
        name, src = bench.kernel_label(*args)
        assert os.path.exists(os.path.join(bench.ROOT, "paper_1101_3615_gb300", "csrc", src))


def test_committed_traffic_is_keyed_by_source_and_variant():
    with open(os.path.join(bench.ROOT, "profiles", "ncu_traffic.json")) as f:
        e = json.load(f)["fwd_born"]
    fresh = e["source_sha"] == bench.kernel_source_hash(e["source"]) and all(
        bench.kernel_source_hash(f) == h for f, h in e.get("deps", {}).items())
    got = bench.ncu_traffic("fwd_born", e["source"], dict(e["variant"]))
    assert got == (float(e["dram_bytes_per_launch"]) if fresh else None)
    other = {k: (v + 1 if isinstance(v, int) else v) for k, v in e["variant"].items()}
    assert bench.ncu_traffic("fwd_born", e["source"], other) is None
    assert bench.ncu_traffic("fwd_born", "stencil2d.cu", dict(e["variant"])) is None
    for f, h in e.get("deps", {}).items():
        assert len(h) == 16 and os.path.exists(os.path.join(bench.ROOT, "paper_1101_3615_gb300", "csrc", f))
    assert abs(e["dram_bytes_read_per_launch"] + e["dram_bytes_write_per_launch"]
               - e["dram_bytes_per_launch"]) < 1.0
