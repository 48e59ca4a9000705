"""The ncu summaries under profiles/ are short text: each gives the command that made it, every ncu
command leaves the GPU clocks alone (--clock-control none), and each command runs committed files only."""
import pathlib
import re

ROOT = pathlib.Path(__file__).resolve().parents[1]
PROFILES = ROOT / "profiles"


def _commands(text):
    # join shell continuation lines, then keep the lines that run ncu
    joined = re.sub(r"\\\n\s*", " ", text)
    return [ln.strip() for ln in joined.splitlines() if re.match(r"\s*(\S+=\S+\s+)*ncu\s", ln)]


def test_profiles_are_short_text_summaries():
    files = sorted(PROFILES.iterdir())
    assert files
    for f in files:
        assert f.suffix in (".md", ".txt", ".json"), f.name
        assert f.stat().st_size < 16 * 1024, f.name


def test_every_ncu_command_keeps_the_clocks_and_runs_committed_files():
    seen = 0
    for f in sorted(PROFILES.glob("*.md")):
        text = f.read_text()
        cmds = _commands(text)
        assert cmds, f"{f.name} gives no ncu command"
        for c in cmds:
            seen += 1
            assert "--clock-control none" in c, (f.name, c)
            for script in re.findall(r"python3?\s+(\S+\.py)", c):
                assert (ROOT / script).is_file(), (f.name, script)
            assert "_work" not in c, (f.name, c)
    assert seen >= 10
