"""Every ncu summary under profiles/ is short text that gives the full command
it came from; every ncu command there keeps the GPU clocks untouched
(--clock-control none) and runs committed files only."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PROFILES = os.path.join(ROOT, "profiles")


def _files():
    return sorted(f for f in os.listdir(PROFILES) if not f.startswith("."))


def test_profiles_are_short_text():
    files = _files()
    assert files
    for f in files:
        assert f.endswith((".md", ".txt")), f
        assert os.path.getsize(os.path.join(PROFILES, f)) < 16 * 1024, f


def test_every_summary_gives_its_ncu_command():
    for f in _files():
        text = open(os.path.join(PROFILES, f)).read()
        blocks = re.findall(r"```(.*?)```", text, flags=re.S)
        cmds = [b for b in blocks if "ncu " in b]
        assert cmds, f"{f}: no ncu command"
        for b in cmds:
            joined = b.replace("\\\n", " ")
            for line in joined.splitlines():
                if re.search(r"\bncu\b", line):
                    assert "--clock-control none" in line, (f, line)
            # the programs it runs are committed files of this repository
            for script in re.findall(r"python3? ([\w/.-]+\.py)", joined):
                assert os.path.exists(os.path.join(ROOT, script)), (f, script)
            assert "_work/" not in joined, f
