"""The product path has no CPU fallback and never touches the oracle (CPU
checks): without libgrom.so every call raises, and no file of the package
imports the oracle or the input generators."""
import ast
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2311_03694_gb300")


def test_calls_raise_without_the_library(tmp_path):
    code = (
        "import sys; sys.path.insert(0, %r)\n"
        "import numpy as np\n"
        "import paper_2311_03694_gb300 as grom\n"
        "grom._build_mod.LIB = %r\n"
        "for call in (lambda: grom.load(), lambda: grom.max_n('full', 'f64'),\n"
        "             lambda: grom.Rom(4, 'full', 'f64', tensor=np.zeros((4, 4, 4)), stiffness=np.ones(4)),\n"
        "             lambda: grom.tune_space('full', 'bf16', 64, 16)):\n"
        "    try:\n"
        "        call()\n"
        "    except RuntimeError as e:\n"
        "        assert 'not built' in str(e), e\n"
        "    else:\n"
        "        raise SystemExit('a call succeeded without the library')\n"
        "print('raised')\n" % (ROOT, str(tmp_path / "missing" / "libgrom.so")))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and "raised" in r.stdout, r.stdout + r.stderr


def test_package_never_imports_the_oracle_or_the_generators():
    for dirpath, _, files in os.walk(PKG):
        for f in files:
            if not f.endswith(".py"):
                continue
            tree = ast.parse(open(os.path.join(dirpath, f)).read())
            for node in ast.walk(tree):
                names = []
                if isinstance(node, ast.Import):
                    names = [a.name for a in node.names]
                elif isinstance(node, ast.ImportFrom) and node.module:
                    names = [node.module]
                for nm in names:
                    assert nm.split(".")[0] not in ("oracle", "synth"), (f, nm)


def test_native_sources_never_reference_the_oracle():
    csrc = os.path.join(PKG, "csrc")
    for f in os.listdir(csrc):
        src = open(os.path.join(csrc, f), errors="replace").read()
        assert "oracle" not in src.lower(), f
