"""The committed ncu summaries: every `ncu` command they quote leaves the
GPU clocks alone (`--clock-control none`), and every stored traffic record
names its command and a source hash (the bench reports its bytes only while
the hash matches the kernel's sources)."""
import glob
import json
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def ncu_commands(text):
    # a command may continue over lines ending in a backslash
    joined = re.sub(r"\\\n\s*", " ", text)
    return [line for line in joined.splitlines() if re.search(r"(^|\s)ncu\s+--", line)]


def test_every_quoted_ncu_command_keeps_the_clocks():
    files = glob.glob(os.path.join(ROOT, "profiles", "*.md"))
    assert files
    for f in files:
        with open(f) as fh:
            for cmd in ncu_commands(fh.read()):
                assert "--clock-control none" in cmd, (os.path.basename(f), cmd)


def test_traffic_records_name_command_and_hash():
    files = glob.glob(os.path.join(ROOT, "profiles", "*_traffic.json"))
    assert files
    for f in files:
        with open(f) as fh:
            d = json.load(fh)
        assert d["dram_bytes_per_launch"] == d["dram_read_bytes"] + d["dram_write_bytes"]
        assert "--clock-control none" in d["command"] and d["command"].startswith("ncu ")
        assert re.fullmatch(r"[0-9a-f]{16}", d["src_hash"])
