"""The committed evidence under profiles/ is text only, its commands run committed files only,
and every DRAM-traffic record that bench.py reads is well formed."""
import json
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PROFILES = os.path.join(ROOT, "profiles")


def test_profiles_are_short_text_files():
    for f in os.listdir(PROFILES):
        path = os.path.join(PROFILES, f)
        assert f.endswith((".md", ".txt", ".json")), f
        assert os.path.getsize(path) < 64 * 1024, f


def test_profile_commands_run_committed_files_only():
    for f in os.listdir(PROFILES):
        if not f.endswith(".md"):
            continue
        text = open(os.path.join(PROFILES, f)).read()
        assert "_work" not in text and "/root" not in text, f
        for script in re.findall(r"python\s+(\S+\.py)", text):
            assert os.path.exists(os.path.join(ROOT, script)), (f, script)


def test_traffic_records_cover_the_keys_bench_reads():
    records = json.load(open(os.path.join(PROFILES, "traffic.json")))
    bench = open(os.path.join(ROOT, "bench.py")).read()
    keys = set(re.findall(r'traffic_per_unit\("([^"]+)"\)', bench))
    keys |= {"select_kernel/n%d" % n for n in (1 << 22, 1 << 18)}   # the f-string keys of the selection leg
    assert keys, "bench.py reads no traffic records"
    for k in keys:
        assert k in records, k
        rec = records[k]
        assert rec["dram_bytes"] > 0 and rec["units"] > 0, k
        assert re.fullmatch(r"[0-9a-f]{16}", rec["engine_sha"]), k
