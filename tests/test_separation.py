"""The oracle and the CUDA library stay independent (read from the sources, no
GPU): nothing under the package or the input generators imports, loads or
includes anything of the oracle, and the oracle neither imports the package
nor loads its library. Only the tests, the smoke check and the benchmark's
CPU-baseline leg use the oracle."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _sources(top, exts):
    for d, _, files in os.walk(os.path.join(ROOT, top)):
        if "_build" in d or "__pycache__" in d:
            continue
        for f in files:
            if f.endswith(exts):
                yield os.path.join(d, f)


def _code(path):
    """The file without its comments and docstrings."""
    text = open(path, encoding="utf-8").read()
    if path.endswith(".py"):
        text = re.sub(r'"""[\s\S]*?"""', "", text)
        return "\n".join(line.split("#", 1)[0] for line in text.splitlines())
    text = re.sub(r"/\*[\s\S]*?\*/", "", text)
    return "\n".join(line.split("//", 1)[0] for line in text.splitlines())


def test_library_and_generators_never_touch_the_oracle():
    exts = (".py", ".cu", ".cuh", ".h", ".c", ".cpp")
    for top in ("paper_2309_03308_gb300", "gen", "include"):
        for path in _sources(top, exts):
            code = _code(path)
            assert not re.search(r"\boracle\b", code), path
            assert "liboracle" not in code, path


def test_oracle_never_touches_the_library():
    for path in _sources("oracle", (".py", ".c", ".h")):
        code = _code(path)
        assert "paper_2309_03308_gb300" not in code, path
        assert "libccorr" not in code, path
        assert "ccorr.h" not in code, path
