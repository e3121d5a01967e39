"""The C ABI from C: `tests/c_client/fft_file.c` includes only wsfft.h and the
CUDA runtime, allocates with cudaMalloc, and runs wsfft_plan_create /
wsfft_execute / wsfft_plan_sync_status / wsfft_destroy.  On the CPU the
client is compiled and linked against the built library (the header is C,
the symbols resolve); on a GPU it transforms seeded arrays read from a file,
and its output is compared with the FP64 oracle."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_2209_15040_gb300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "c_client", "fft_file.c")
CUDA = os.environ.get("CUDA_HOME", "/usr/local/cuda")


def _compile(out_dir):
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    lib = build.build_library()
    exe = os.path.join(out_dir, "fft_file")
    libdir = os.path.dirname(lib)
    cmd = [gcc, "-std=c11", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
           "-I", os.path.join(CUDA, "include"), SRC, "-o", exe,
           "-L", libdir, "-lwsfft", "-Wl,-rpath," + libdir,
           "-L", os.path.join(CUDA, "lib64"), "-lcudart", "-Wl,-rpath," + os.path.join(CUDA, "lib64")]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return exe


def test_c_client_compiles_and_links(tmp_path):
    exe = _compile(str(tmp_path))
    assert os.path.exists(exe)


CODES = {"c32": 0, "c16f": 1, "c16bf": 2}
TOLS = {"c32": 5e-6, "c16f": 3e-3, "c16bf": 2e-2}


@pytest.mark.gpu
@pytest.mark.parametrize("dims,batch,direction,dtype", [((64, 32, 16), 2, -1, "c32"), ((1 << 14,), 3, 1, "c32"),
                                                        ((128, 256), 1, -1, "c32"), ((512, 512, 512), 1, -1, "c32"),
                                                        ((64, 64, 64), 2, -1, "c16f"), ((128, 512), 1, 1, "c16bf")])
def test_c_client_matches_oracle(tmp_path, dims, batch, direction, dtype):
    import oracle
    from paper_2209_15040_gb300 import inputs
    exe = _compile(str(tmp_path))
    dist = "normal" if dtype == "c32" else "uniform"
    xs = np.ascontiguousarray(inputs.complex_input((batch,) + dims, 81, dist, dtype))
    fin, fout = str(tmp_path / "in.bin"), str(tmp_path / "out.bin")
    xs.tofile(fin)
    r = subprocess.run([exe, fin, fout, str(CODES[dtype]), str(direction), str(batch)] + [str(d) for d in dims],
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr
    got = np.fromfile(fout, dtype=xs.dtype).reshape(xs.shape)
    got = inputs.storage_to_c128(got, dtype)
    # the library's default normalisation: paper for complex64, orthonormal for 16-bit storage
    norm = oracle.NORM_PAPER if dtype == "c32" else oracle.NORM_ORTHO
    ref = oracle.fftn(inputs.storage_to_c128(xs, dtype), rank=len(dims), sign=direction, norm=norm)
    err = oracle.rel_l2(got, ref)
    print(f"C client {dims} x{batch} {dtype} direction {direction}: rel_l2 {err:.2e}")
    assert err < TOLS[dtype]
