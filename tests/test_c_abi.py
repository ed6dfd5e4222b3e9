"""The boundary is a C ABI: a C99 program that includes include/whff.h compiles
with warnings as errors, links against the library and runs the host-side
calls (no GPU needed): sizes, the fixed-rate and fixed-accuracy encoders,
refusals with their codes and messages, and the version string."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

C_SOURCE = r"""
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "whff.h"

int main(void) {
  const int64_t M = 9, N = 13;
  double A[9 * 13];
  for (int i = 0; i < 9; ++i)
    for (int j = 0; j < 13; ++j) A[i * 13 + j] = exp(-0.1 * (double)((i - j) * (i - j)));
  /* fixed-rate WZ2 at rate 16: 64 + ceil(9/4) * ceil(13/4) * 32 bytes */
  size_t cap = whff_compressed_size(WHFF_FMT_FIXED_LIFT, 16, M, N), len = 0;
  if (cap != 64 + 3 * 4 * 32) return 1;
  unsigned char* blob = (unsigned char*)malloc(cap);
  if (whff_compress(A, M, N, N, WHFF_FMT_FIXED_LIFT, 16, blob, cap, &len, 1) != WHFF_OK || len != cap) return 2;
  if (memcmp(blob, "WZ1", 4) != 0) return 3;
  /* refusals: rate outside 8..24, an oversized shape, a non-finite entry */
  if (whff_compress(A, M, N, N, WHFF_FMT_FIXED_LIFT, 28, blob, cap, &len, 1) != WHFF_EINVAL) return 4;
  if (whff_compressed_size(WHFF_FMT_FIXED_LIFT, 16, (int64_t)1 << 50, 4) != 0) return 5;
  A[5] = NAN;
  if (whff_compress(A, M, N, N, WHFF_FMT_FIXED_LIFT, 16, blob, cap, &len, 1) != WHFF_ENONFINITE) return 6;
  if (strlen(whff_last_error()) == 0) return 7;
  A[5] = 0.5;
  /* fixed accuracy: at most whff_accuracy_max_size bytes */
  size_t acap = whff_accuracy_max_size(M, N), alen = 0;
  unsigned char* acc = (unsigned char*)malloc(acap);
  if (whff_compress_accuracy(A, M, N, N, 1e-6, acc, acap, &alen, 0) != WHFF_OK || alen == 0 || alen > acap) return 8;
  if (whff_compress_accuracy(A, M, N, N, -1.0, acc, acap, &alen, 0) != WHFF_EINVAL) return 9;
  printf("%zu %zu %s\n", len, alen, whff_version());
  free(blob);
  free(acc);
  return 0;
}
"""


def test_c_program_uses_the_abi(tmp_path):
    import paper_1902_08018_gb300 as W

    W.library()  # built and up to date
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "abi.c"
    src.write_text(C_SOURCE)
    exe = tmp_path / "abi"
    libdir = os.path.join(ROOT, "paper_1902_08018_gb300")
    cmd = [gcc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"), str(src),
           "-L", libdir, "-lwhff", f"-Wl,-rpath,{libdir}", "-lm", "-o", str(exe)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, (r.returncode, r.stdout, r.stderr)
    blob_len, acc_len, version = r.stdout.split(maxsplit=2)
    assert version.startswith("whff") and int(blob_len) == 64 + 3 * 4 * 32 and int(acc_len) > 64
