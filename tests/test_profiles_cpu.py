"""The committed ncu summaries: every one cited by the documentation exists, and every
command in them leaves the GPU clocks alone (--clock-control none) and runs committed
files only."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PROFILES = os.path.join(ROOT, "profiles")


def _docs():
    text = ""
    for name in ("DESIGN.md", "README.md"):
        path = os.path.join(ROOT, name)
        if os.path.exists(path):
            with open(path) as f:
                text += f.read()
    return text


def test_cited_profiles_exist():
    cited = set(re.findall(r"profiles/([A-Za-z0-9_.\-]+\.md)", _docs()))
    assert cited, "the documentation cites no profile"
    missing = sorted(c for c in cited if not os.path.exists(os.path.join(PROFILES, c)))
    assert not missing, missing


def test_profile_commands_leave_clocks_alone():
    for name in sorted(os.listdir(PROFILES)):
        if not name.endswith(".md"):
            continue
        with open(os.path.join(PROFILES, name)) as f:
            text = f.read()
        # an ncu invocation starts a command line (possibly indented), not a sentence
        for m in re.finditer(r"(?m)^\s*ncu\s(?:[^\n]*\\\n)*[^\n]*", text):
            cmd = m.group(0)
            assert "--clock-control none" in cmd, (name, cmd)
            assert "_work/" not in cmd, (name, cmd)
