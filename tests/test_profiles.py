"""The ncu summaries under profiles/ (CPU checks): each gives the command that
made it, with ncu's clock control off, and that command runs committed files
only (no working files, no scratch scripts)."""
import json
import os
import re
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PROF = os.path.join(ROOT, "profiles")


def _tracked():
    out = subprocess.run(["git", "ls-files"], cwd=ROOT, capture_output=True, text=True)
    return set(out.stdout.split()) if out.returncode == 0 else None


def _commands():
    for f in sorted(os.listdir(PROF)):
        path = os.path.join(PROF, f)
        text = open(path).read()
        if f.endswith(".json"):
            for ent in json.load(open(path)).values():
                yield f, ent["command"]
        else:
            # a command: lines from "ncu" (or "python") through their backslash continuations
            lines = text.splitlines()
            i = 0
            while i < len(lines):
                ln = lines[i].strip()
                if ln.startswith("ncu ") or ln.startswith("python "):
                    cmd = [ln]
                    while cmd[-1].endswith("\\") and i + 1 < len(lines):
                        i += 1
                        cmd.append(lines[i].strip())
                    yield f, " ".join(c.rstrip("\\").strip() for c in cmd)
                i += 1


def test_every_summary_gives_its_command():
    files = [f for f in os.listdir(PROF) if f.endswith(".md")]
    assert files
    for f in files:
        assert any(name == f for name, _ in _commands()), f


def test_commands_run_committed_files_with_clock_control_off():
    tracked = _tracked()
    seen = 0
    for f, cmd in _commands():
        if cmd.startswith("ncu "):
            assert "--clock-control none" in cmd, (f, cmd)
        for script in re.findall(r"python ([\w./-]+\.py)", cmd):
            seen += 1
            assert not script.startswith("_work"), (f, script)
            assert os.path.exists(os.path.join(ROOT, script)), (f, script)
            if tracked is not None:
                assert script in tracked, (f, script)
    assert seen > 0
