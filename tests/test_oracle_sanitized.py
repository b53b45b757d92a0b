"""The FP64 oracle under AddressSanitizer and UndefinedBehaviorSanitizer.

tests/oracle_sanitize_driver.c runs every entry point of oracle/eik_oracle.c on
small grids with the method's edge cases (single nodes and lines, shapes that are
not multiples of a tile, impassable nodes, duplicated or missing sources, a
source out of range, unequal spacings) and checks that fast marching,
Gauss-Seidel sweeping, Algorithm 2 and the FIM agree.  Built with the oracle's
own flags plus -fsanitize=address,undefined and no recovery, it must exit 0: no
out-of-bounds access, use after free, leak or undefined behaviour on these paths.
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_oracle_under_address_and_undefined_behaviour_sanitizers(tmp_path):
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not available")
    exe = str(tmp_path / "oracle_sanitize_driver")
    subprocess.check_call([gcc, "-O1", "-g", "-std=c11", "-fno-fast-math", "-ffp-contract=off",
                           "-fsanitize=address,undefined", "-fno-sanitize-recover=all", "-fno-omit-frame-pointer",
                           os.path.join(ROOT, "oracle", "eik_oracle.c"),
                           os.path.join(ROOT, "tests", "oracle_sanitize_driver.c"), "-lm", "-o", exe])
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=1", UBSAN_OPTIONS="print_stacktrace=1:halt_on_error=1")
    p = subprocess.run([exe], capture_output=True, text=True, env=env, timeout=600)
    assert p.returncode == 0, p.stderr[-4000:]
    assert "oracle sanitize driver ok" in p.stdout
