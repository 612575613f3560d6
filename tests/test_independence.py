"""The oracle and the CUDA path stay independent (CPU only, static checks).

* no module of the library package imports the oracle, the tests or bench.py,
  and no oracle module imports the library package;
* the seeded input generators shared by both sides import nothing but math
  and numpy (they hold none of the method's arithmetic);
* the CUDA sources include nothing from the oracle or the tests;
* nothing committed refers to the untracked working folder;
* the binding refuses to run without a CUDA device instead of falling back
  to any CPU path.
"""
import ast
import glob
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, 'paper_2003_01490_gb300')


def imported_modules(path):
    """Top-level names of every module a Python file imports, at any depth."""
    tree = ast.parse(open(path).read(), filename=path)
    names = set()
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            names.update(a.name.split('.')[0] for a in node.names)
        elif isinstance(node, ast.ImportFrom):
            if node.level == 0 and node.module:
                names.add(node.module.split('.')[0])
            elif node.level > 0:
                names.add('.')
    return names


def test_library_never_imports_the_oracle():
    for path in glob.glob(os.path.join(PKG, '*.py')):
        bad = imported_modules(path) & {'oracle', 'tests', 'cases', 'bench', '__graft_entry__'}
        assert not bad, (path, bad)


def test_oracle_never_imports_the_library():
    for path in glob.glob(os.path.join(ROOT, 'oracle', '*.py')):
        bad = imported_modules(path) & {'paper_2003_01490_gb300', 'bench', 'tests', 'cases', 'torch',
                                        'ctypes'}
        assert not bad, (path, bad)


def test_shared_input_generators_hold_no_method_code():
    assert imported_modules(os.path.join(PKG, 'workloads.py')) <= {'math', 'numpy'}


def test_cuda_sources_include_only_their_own_headers():
    for path in glob.glob(os.path.join(PKG, 'csrc', '*')):
        for line in open(path):
            if line.lstrip().startswith('#include'):
                assert 'oracle' not in line and 'tests' not in line, (path, line)


def test_nothing_committed_refers_to_the_working_folder():
    try:
        files = subprocess.run(['git', 'ls-files'], cwd=ROOT, capture_output=True, text=True,
                               check=True).stdout.split()
    except (OSError, subprocess.CalledProcessError):
        pytest.skip('not a git checkout')
    here = os.path.relpath(__file__, ROOT)
    for f in files:
        if f == here or not f.endswith(('.py', '.cu', '.cuh', '.h', '.c', '.sh')):
            continue
        text = open(os.path.join(ROOT, f), errors='replace').read()
        assert '_work/' not in text and "'_work'" not in text, f


def test_binding_refuses_to_run_without_cuda():
    torch = pytest.importorskip('torch')
    if torch.cuda.is_available():
        pytest.skip('a CUDA device is present')
    from paper_2003_01490_gb300 import build, lbmdem
    if not os.path.exists(lbmdem.LIB_PATH):
        build.build()
    r, d = lbmdem.lbm_default_params()
    with pytest.raises(RuntimeError, match='CUDA device required'):
        lbmdem.lbm_create(lbmdem.make_grid((16, 16, 16)), r, (0, 0, 0), d, 'f32', 1)
