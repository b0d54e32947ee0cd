"""The library and its binding never reach the oracle: no source file of the package names it,
and importing the binding (and the training driver) loads no oracle module. The oracle is test
infrastructure; the only path from the package to results is libsem.so."""
import os
import re
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1506_05996_gb300")


def _sources():
    for base, dirs, files in os.walk(PKG):
        dirs[:] = [d for d in dirs if d not in ("_build", "__pycache__")]
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                yield os.path.join(base, f)


def test_no_package_source_imports_or_includes_the_oracle():
    py_import = re.compile(r"^\s*(import\s+oracle\b|from\s+oracle\b)", re.M)
    c_include = re.compile(r'#\s*include\s*[<"][^">]*oracle', re.M)
    checked = 0
    for path in _sources():
        src = open(path, encoding="utf-8").read()
        assert not py_import.search(src), path
        assert not c_include.search(src), path
        assert "oracle/" not in src, path
        checked += 1
    assert checked >= 10


def test_importing_the_binding_loads_no_oracle_module():
    code = ("import sys; import paper_1506_05996_gb300.sem, paper_1506_05996_gb300.learn; "
            "print(sorted(m for m in sys.modules if m == 'oracle' or m.startswith('oracle.')))")
    out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    assert out.stdout.strip().splitlines()[-1] == "[]"


def test_binding_without_the_library_fails_loudly(tmp_path):
    """With libsem.so absent the binding refuses to import: there is no fallback path."""
    import shutil
    pkg = tmp_path / "paper_1506_05996_gb300"
    pkg.mkdir()
    shutil.copy(os.path.join(PKG, "__init__.py"), pkg / "__init__.py")
    shutil.copy(os.path.join(PKG, "sem.py"), pkg / "sem.py")
    code = "import paper_1506_05996_gb300.sem"
    out = subprocess.run([sys.executable, "-c", code], cwd=str(tmp_path), capture_output=True, text=True,
                         timeout=300, env={**os.environ, "PYTHONPATH": str(tmp_path)})
    assert out.returncode != 0
    assert "libsem.so is not built" in out.stderr
