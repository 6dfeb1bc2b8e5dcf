"""The commands quoted in profiles/ still run against the committed files:
every `python bench.py ...` parses with bench.py's own command line, every
`ncu -k regex:NAME` names a kernel defined in the CUDA sources, and no command
runs anything outside the repository's committed files."""
import importlib.util
import re
import shlex
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]
PROFILES = sorted((ROOT / "profiles").glob("*.md"))
CSRC = ROOT / "paper_1807_08084_gb300" / "csrc"
STOP = {">", ">>", "&&", "||", "|", ";", "2>&1", "&"}


def _bench_parser():
    spec = importlib.util.spec_from_file_location("bench_cli", ROOT / "bench.py")
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod.build_parser()


def _commands(md: Path):
    """Shell commands of the file's code blocks, continuation lines joined."""
    blocks = re.findall(r"```[a-z]*\n(.*?)```", md.read_text(), flags=re.S)
    for block in blocks:
        text = re.sub(r"\\\n\s*", " ", block)
        for line in text.splitlines():
            if line.strip():
                yield line.strip()


def _after(tokens, i):
    out = []
    for t in tokens[i + 1:]:
        if t in STOP or t.startswith(">") or t.startswith("2>"):
            break
        out.append(t)
    return out


def _kernel_names():
    src = "\n".join(p.read_text() for p in CSRC.glob("*.cu*"))
    bounds = r"__launch_bounds__\((?:[^()]|\([^()]*\))*\)\s*"  # one level of nested calls
    return set(re.findall(r"__global__\s+void\s+(?:" + bounds + r")?(\w+)\s*\(", src))


def test_profiles_have_commands():
    assert PROFILES
    assert any("bench.py" in c for md in PROFILES for c in _commands(md))


@pytest.mark.parametrize("md", PROFILES, ids=lambda p: p.name)
def test_profile_commands_run_committed_files(md):
    parser = _bench_parser()
    kernels = _kernel_names()
    assert kernels, "no kernels found in the CUDA sources"
    for cmd in _commands(md):
        assert "_work/" not in cmd, f"{md.name}: {cmd}"
        tokens = shlex.split(cmd)
        for i, t in enumerate(tokens):
            if t.endswith("bench.py"):
                parser.parse_args(_after(tokens, i))  # SystemExit on an unknown flag
            if t == "-k" and i + 1 < len(tokens) and tokens[i + 1].startswith("regex:"):
                name = tokens[i + 1][len("regex:"):]
                assert any(re.search(name, k) for k in kernels), f"{md.name}: no kernel {name}"
