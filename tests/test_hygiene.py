"""Source hygiene checks that need no GPU: no source names the CUDA batched
copy entry points (they are not used anywhere in this library), and code
and comments stand on their own (no pointers into planning documents or
machine paths)."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SOURCE_DIRS = ["paper_1308_2864_gb300", "include", "oracle", "ks_inputs", "tests"]
SOURCE_FILES = ["bench.py", "__graft_entry__.py"]
EXTS = (".py", ".cu", ".cuh", ".h", ".c", ".cpp", ".sh")


def sources():
    for f in SOURCE_FILES:
        yield os.path.join(ROOT, f)
    for d in SOURCE_DIRS:
        for dirpath, dirnames, files in os.walk(os.path.join(ROOT, d)):
            dirnames[:] = [x for x in dirnames if x not in ("lib", "__pycache__")]
            for f in files:
                if f.endswith(EXTS):
                    yield os.path.join(dirpath, f)


def test_no_batched_copy_entry_points():
    names = [pre + "emcpy" + mid + "BatchAsync" for pre in ("cudaM", "cuM") for mid in ("", "3D")]
    for path in sources():
        txt = open(path, encoding="utf-8").read()
        for name in names:
            assert name not in txt, f"{path} names {name}"


def test_code_does_not_point_into_planning_documents():
    words = ["SURVEY", "DESIGN" + ".md", "BASELINE" + ".json", "BASELINE" + ".md", "VERDICT",
             "ADVICE" + ".md", "north" + "_star", "gpu" + "run", "/root" + "/", "configs" + "[",
             "_work" + "/"]
    me = os.path.abspath(__file__)
    for path in sources():
        if os.path.abspath(path) == me:
            continue
        txt = open(path, encoding="utf-8").read()
        for w in words:
            assert w not in txt, f"{path} mentions {w}"


def test_oracle_is_imported_only_by_test_infrastructure():
    # the product package and the input generators never import the oracle;
    # bench.py and __graft_entry__.py may (cpu_baseline / smoke)
    pat = re.compile(r"^\s*(from\s+oracle\b|import\s+oracle\b)", re.M)
    for d in ("paper_1308_2864_gb300", "ks_inputs", "include"):
        for dirpath, _, files in os.walk(os.path.join(ROOT, d)):
            for f in files:
                if f.endswith(EXTS):
                    txt = open(os.path.join(dirpath, f), encoding="utf-8").read()
                    assert not pat.search(txt), os.path.join(dirpath, f)
