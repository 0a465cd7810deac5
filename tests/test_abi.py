"""Host-side checks of the C ABI: the library builds for sm_103a and exports
every entry point include/ch.h declares (no device calls)."""
import ctypes as C
import os
import re
import subprocess

import pytest

from paper_2412_18008_gb300 import build as B

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                      "include", "ch.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(ch_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_entry_points():
    names = declared_functions()
    for must in ("ch_build", "ch_query_batch", "ch_query_batch_host", "ch_free",
                 "ch_export", "ch_get_stats", "ch_last_error"):
        assert must in names


def test_library_builds_and_exports_every_symbol():
    lib_path = B.build()
    assert os.path.exists(lib_path)
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (ch_\w+)", out))
    missing = [f for f in declared_functions() if f not in exported]
    assert not missing, missing


def test_library_loads_and_reports_version():
    lib = C.CDLL(B.build())
    lib.ch_version.restype = C.c_char_p
    assert b"sm_103a" in lib.ch_version()


def test_struct_layouts_match_header():
    from paper_2412_18008_gb300 import ch
    # offsets of the C structs, computed by the host compiler from ch.h
    src = r'''
    #include <stddef.h>
    #include <stdio.h>
    #include "ch.h"
    int main(void) {
      printf("%zu %zu %zu\n", sizeof(ch_graph_t), sizeof(ch_params_t), sizeof(ch_stats_t));
      printf("%zu %zu\n", offsetof(ch_params_t, stream), offsetof(ch_stats_t, witness_bytes));
      printf("%zu %zu %zu\n", sizeof(ch_query_config_t), sizeof(ch_server_params_t),
             offsetof(ch_server_params_t, idle_ms));
      return 0;
    }'''
    tmp = "/tmp/ch_layout_check"
    with open(tmp + ".c", "w") as f:
        f.write(src)
    subprocess.run(["gcc", "-I", os.path.dirname(HEADER), tmp + ".c", "-o", tmp], check=True)
    vals = subprocess.run([tmp], capture_output=True, text=True, check=True).stdout.split()
    sizes = list(map(int, vals))
    assert sizes[0] == C.sizeof(ch.GraphT)
    assert sizes[1] == C.sizeof(ch.ParamsT)
    assert sizes[2] == C.sizeof(ch.StatsT)
    assert sizes[3] == ch.ParamsT.stream.offset
    assert sizes[4] == ch.StatsT.witness_bytes.offset
    assert sizes[5] == C.sizeof(ch.QueryConfigT)
    assert sizes[6] == C.sizeof(ch.ServerParamsT)
    assert sizes[7] == ch.ServerParamsT.idle_ms.offset


def test_autotune_candidates_match_the_header():
    # the binding's candidate list has the header's length and its order:
    # 4 * small_first + 2 * warp layout + (threads == 256) without stalling,
    # then the stalling warp layout, then the delta candidates
    from paper_2412_18008_gb300 import ch
    text = open(HEADER).read()
    n = int(re.search(r"#define CH_QUERY_AUTOTUNE_CONFIGS (\d+)", text).group(1))
    assert len(ch.QUERY_CONFIGS) == n
    for i, (lay, thr, sf, stall, delta) in enumerate(ch.QUERY_CONFIGS[:8]):
        assert i == 4 * sf + 2 * lay + (thr == 256) and stall == 0 and delta == 0
    for i, (lay, thr, sf, stall, delta) in enumerate(ch.QUERY_CONFIGS[8:12]):
        assert i == 2 * sf + (thr == 256) and lay == ch.CH_QUERY_WARP_FLAT and stall == 1 and delta == 0
    tail = ch.QUERY_CONFIGS[12:]
    assert all(c[:4] == (ch.CH_QUERY_WARP_FLAT, 256, 1, 1) and c[4] > 0 for c in tail)
    mults = re.search(r"delta = ([\d, ]+) x the weight scale", " ".join(text.split())).group(1)
    assert [c[4] for c in tail] == [int(x) for x in mults.split(",")]
    src = open(os.path.join(os.path.dirname(HEADER), "..", "paper_2412_18008_gb300", "csrc", "query.cu")).read()
    lib_mults = re.search(r"DELTA_TUNE_MULT\[\d+\] = \{([\d, ]+)\}", src).group(1)
    assert [c[4] for c in tail] == [int(x) for x in lib_mults.split(",")]


def test_no_cpu_fallback_in_product_package():
    pkg = os.path.join(os.path.dirname(HEADER), "..", "paper_2412_18008_gb300")
    for root, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh")):
                text = open(os.path.join(root, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f


def test_bench_touches_the_oracle_only_in_its_baseline_legs():
    # bench.py may run the oracle only to time it: the cpu_baseline record
    # and the reference arm (through oracle_build_s)
    import ast
    path = os.path.join(os.path.dirname(HEADER), "..", "bench.py")
    tree = ast.parse(open(path).read())
    allowed = {"oracle_build_s", "cpu_baseline_record", "run_reference"}
    users = set()
    for fn in ast.walk(tree):
        if not isinstance(fn, ast.FunctionDef):
            continue
        for node in ast.walk(fn):
            if isinstance(node, (ast.Import, ast.ImportFrom)):
                mods = [a.name for a in node.names] if isinstance(node, ast.Import) else [node.module or ""]
                if any(m == "oracle" or m.startswith("oracle.") for m in mods):
                    users.add(fn.name)
            if isinstance(node, ast.Call) and isinstance(node.func, ast.Name) and node.func.id == "oracle_build_s":
                users.add(fn.name)
    assert users and users <= allowed, users - allowed
    top = [n for n in tree.body if isinstance(n, (ast.Import, ast.ImportFrom))]
    assert not any((a.name if isinstance(n, ast.Import) else n.module or "").startswith("oracle")
                   for n in top for a in n.names), "bench.py imports the oracle at module level"


def test_device_code_has_no_trap_or_device_assert():
    # failures inside kernels are reported through error words the host
    # reads, never by trapping the GPU
    csrc = os.path.join(os.path.dirname(HEADER), "..", "paper_2412_18008_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        if f.endswith((".cu", ".cuh")):
            text = re.sub(r"//[^\n]*|/\*.*?\*/", "", open(os.path.join(csrc, f)).read(), flags=re.S)
            assert "__trap" not in text and "brkpt" not in text, f
            assert not re.search(r"(?<![\w_])assert\s*\(", text), f
