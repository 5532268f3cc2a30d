"""Builds and runs the CPU oracle (oracle/inet_oracle.cpp) for the tests.

Test infrastructure: the oracle is a separate executable with its own parser;
nothing here is shared with the CUDA path.
"""
from __future__ import annotations

import json
import os
import subprocess
import tempfile

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "inet_oracle.cpp")
BIN = os.path.join(ROOT, "oracle", "inet_oracle")


def compile_oracle(out: str, src: str = SRC) -> str:
    subprocess.run(["g++", "-O2", "-std=c++17", "-pthread", src, "-o", out], check=True)
    return out


def build(force: bool = False) -> str:
    if force or not os.path.exists(BIN) or os.path.getmtime(BIN) < os.path.getmtime(SRC):
        compile_oracle(BIN)
    return BIN


def run(rules: str, nets: list[str] | str, mode: str = "lifo", seed: int = 1,
        eager: bool = False, threads: int = 1, max_interactions: int | None = None,
        quiet: bool = False, binary: str | None = None, timeout: float = 600) -> list[dict]:
    """Runs the oracle; returns one dict per net (or the rule-set error)."""
    if isinstance(nets, str):
        nets = [nets]
    with tempfile.TemporaryDirectory() as d:
        rp = os.path.join(d, "rules.txt")
        np_ = os.path.join(d, "nets.txt")
        with open(rp, "w") as f:
            f.write(rules)
        with open(np_, "w") as f:
            f.write("\n".join(nets) + "\n")
        cmd = [binary or BIN, rp, np_, "--mode", mode, "--seed", str(seed), "--threads", str(threads)]
        if eager:
            cmd.append("--eager")
        if quiet:
            cmd.append("--quiet")
        if max_interactions is not None:
            cmd += ["--max-interactions", str(max_interactions)]
        p = subprocess.run(cmd, capture_output=True, text=True, timeout=timeout)
    out = [json.loads(line) for line in p.stdout.splitlines() if line.strip()]
    if p.returncode != 0 and not out:
        raise RuntimeError(f"oracle failed ({p.returncode}): {p.stderr[-2000:]}")
    return out
