"""CPU: pieces of the benchmark that need no GPU -- the algorithmic flop count per
value+gradient query against the survey's figures (about 270, 520 and 890 flops at degrees
2, 3 and 4), the per-query window bytes of the decode roofline, and the DRAM-traffic
record, which is reported only for the kernel sources it was captured on."""
import bench


def test_query_flops():
    assert bench.query_flops(3) == 519
    assert bench.query_flops(2) == 270
    assert bench.query_flops(4) == 888
    assert bench.query_flops(3) + bench.RENDER_EXTRA_FLOPS == 559


def test_decode_window_bytes():
    # q rows per support, one load of each z-layer pair's entry (two at degree 3)
    assert bench.DECODE_WINDOW_BYTES[3] == 8 * 32
    assert bench.DECODE_WINDOW_BYTES[2] == 3 * (32 + 16)
    assert bench.DECODE_WINDOW_BYTES[1] == 2 * 16


def test_render_traffic_is_tied_to_the_sources(monkeypatch):
    rec = dict(bench.RENDER_TRAFFIC)
    monkeypatch.setattr(bench, "RENDER_TRAFFIC", dict(rec, src_sha256="0" * 64))
    assert bench.render_traffic() is None                      # sources changed: no number
    monkeypatch.setattr(bench, "RENDER_TRAFFIC", dict(rec, src_sha256=bench.kernel_sources_sha256()))
    assert bench.render_traffic() == rec["bytes_per_launch"]
