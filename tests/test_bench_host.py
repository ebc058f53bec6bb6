"""Host logic of bench.py that needs no GPU: the DRAM-traffic record (taken from an ncu CSV
log, tied to the kernel's source hash, dropped when the source changes) and the oracle run in
independent parts (the parts together make exactly the sample's products)."""
import json

import bench
import oracle
import workloads as W

CSV_HEAD = '"ID","Process ID","Process Name","Host Name","Kernel Name","Context","Stream","Block Size",' \
           '"Grid Size","Device","CC","Section Name","Metric Name","Metric Unit","Metric Value"\n'


def row(i, kernel, metric, unit, value):
    return (f'"{i}","1","python3","h","void {kernel}<3, 0>(int)","1","7","(256, 1, 1)","(608, 1, 1)","0",'
            f'"10.3","Command line profiler metrics","{metric}","{unit}","{value}"\n')


def test_traffic_record_mean_per_launch_and_invalidation(tmp_path, monkeypatch):
    log = tmp_path / "dram.csv"
    log.write_text("==PROF== Connected\n" + CSV_HEAD +
                   row(0, "group_stream_kernel", "dram__bytes_read.sum", "byte", "1,000") +
                   row(0, "group_stream_kernel", "dram__bytes_write.sum", "Kbyte", "2") +
                   row(1, "group_stream_kernel", "dram__bytes_read.sum", "byte", "3000") +
                   row(1, "group_stream_kernel", "dram__bytes_write.sum", "byte", "0") +
                   row(2, "other_kernel", "dram__bytes_read.sum", "byte", "99999"))
    out = tmp_path / "traffic.json"
    monkeypatch.setattr(bench, "source_sha", lambda k: "sha-a")
    bench.record_traffic("plain_large", "group_stream_kernel", str(log), path=str(out))
    entry = json.loads(out.read_text())["plain_large"]
    assert entry["launches"] == 2 and entry["bytes_per_launch"] == (1000 + 2000 + 3000) / 2
    assert bench.ncu_traffic("plain_large", path=str(out)) == ("group_stream_kernel", 3000.0)
    monkeypatch.setattr(bench, "source_sha", lambda k: "sha-b")  # the kernel's sources changed
    assert bench.ncu_traffic("plain_large", path=str(out)) is None
    assert bench.ncu_traffic("imbalanced", path=str(out)) is None


def test_oracle_parts_make_the_whole_sample():
    p = W.plain_small()
    sp, _ = bench.key_sample(p, 3)
    whole = oracle.contract(sp.X, sp.Y, sp.cx, sp.cy, sp.out_order).products
    prods, seconds, desc = bench.run_oracle_parallel(p, "plain_small", 3, 4)
    assert prods == whole and whole > 0 and seconds >= 0
    assert "4 parts" in desc


def test_source_hash_ignores_comments_only(tmp_path, monkeypatch):
    d = tmp_path / "paper_2410_10094_gb300" / "csrc"
    d.mkdir(parents=True)
    f = d / "k.cu"
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "KERNEL_SOURCES", {"k": ["k.cu"]})
    f.write_text("// a kernel\n__global__ void k(int* p) { p[0] = 1; }\n")
    h0 = bench.source_sha("k")
    f.write_text("/* reworded\n   comment */\n__global__ void k(int* p) { p[0] = 1; }  // trailing\n\n")
    assert bench.source_sha("k") == h0
    f.write_text("// a kernel\n__global__ void k(int* p) { p[0] = 2; }\n")
    assert bench.source_sha("k") != h0
