"""The oracle is memory-clean: its C library built with AddressSanitizer and
UndefinedBehaviorSanitizer runs the oracle's pins (all but the Monte-Carlo
estimate, for time) without a report.  Any sanitizer report ends the run
with a non-zero status."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _runtime(name):
    out = subprocess.run(["gcc", f"-print-file-name={name}"], capture_output=True, text=True).stdout.strip()
    return out if os.path.isabs(out) and os.path.exists(out) else None


def test_oracle_pins_under_address_and_ub_sanitizers():
    asan, ubsan = _runtime("libasan.so"), _runtime("libubsan.so")
    if not (asan and ubsan):
        pytest.skip("gcc sanitizer runtimes not found")
    odir = os.path.join(ROOT, "oracle", "_build")
    os.makedirs(odir, exist_ok=True)
    lib = os.path.join(odir, "libvbh_oracle_sanitized.so")
    subprocess.check_call(["gcc", "-O1", "-g", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                           "-fsanitize=address,undefined", "-fno-sanitize-recover=undefined",
                           "-fno-omit-frame-pointer", os.path.join(ROOT, "oracle", "vbh_oracle.c"), "-lm",
                           "-o", lib])
    code = (
        "import os, sys\n"
        f"sys.path.insert(0, {ROOT!r})\n"
        "import oracle.oracle as O\n"
        f"O._LIB = {lib!r}\n"
        "O.build = lambda force=False: O._LIB\n"
        "import pytest\n"
        "rc = pytest.main(['-x', '-q', '-p', 'no:cacheprovider', '-k', 'not monte_carlo',\n"
        f"                 {os.path.join(ROOT, 'tests', 'test_oracle_pins.py')!r},\n"
        f"                 {os.path.join(ROOT, 'tests', 'test_oracle_em_pins.py')!r}])\n"
        "assert O._lib is not None and O._lib._name == O._LIB\n"
        "sys.exit(int(rc))\n")
    env = dict(os.environ, LD_PRELOAD=f"{asan}:{ubsan}", ASAN_OPTIONS="detect_leaks=0",
               UBSAN_OPTIONS="print_stacktrace=1:halt_on_error=1")
    out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True,
                         timeout=900)
    log = out.stdout + out.stderr
    assert out.returncode == 0, log[-3000:]
    assert "runtime error" not in log and "AddressSanitizer" not in log, log[-3000:]
    assert " passed" in log
