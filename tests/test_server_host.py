"""Host logic of the serving loop (queueing, budget admission, first come
first served, rejection, bookkeeping, shutdown) on a mocked CUDA runtime,
under AddressSanitizer and UBSan.  No GPU: server.cu is linked with its CUDA
calls wrapped onto host stand-ins (tests/host_mock/runtime_mock.cpp)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
MOCK = os.path.join(ROOT, "tests", "host_mock")
CSRC = os.path.join(ROOT, "paper_2606_22180_b300", "csrc")
OUT = os.path.join(ROOT, "_build", "host_mock")
WRAPPED = ["cudaMallocAsync", "cudaFreeAsync", "cudaMemcpyAsync", "cudaMemsetAsync", "cudaStreamSynchronize",
           "cudaStreamCreateWithFlags", "cudaStreamDestroy", "cudaGetDevice", "cudaSetDevice"]


@pytest.fixture(scope="module")
def driver():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    os.makedirs(OUT, exist_ok=True)
    san = ["-Xcompiler", "-fsanitize=address", "-Xcompiler", "-fsanitize=undefined"]
    inc = ["-I", os.path.join(ROOT, "include"), "-I", CSRC]
    arch = ["-gencode", "arch=compute_103a,code=sm_103a"]
    subprocess.check_call([nvcc, "-std=c++17", "-g", "-O1", "-x", "cu", "-c", os.path.join(CSRC, "server.cu"),
                           "-o", os.path.join(OUT, "server.o")] + inc + san + arch)
    subprocess.check_call([nvcc, "-std=c++17", "-g", "-O1", "-x", "cu", "-c",
                           os.path.join(MOCK, "runtime_mock.cpp"), "-o", os.path.join(OUT, "runtime_mock.o")]
                          + inc + san)
    subprocess.check_call(["g++", "-std=c++17", "-g", "-O1", "-c", os.path.join(MOCK, "server_driver.cpp"), "-o",
                           os.path.join(OUT, "server_driver.o"), "-I", os.path.join(ROOT, "include"),
                           "-fsanitize=address,undefined"])
    exe = os.path.join(OUT, "server_driver")
    subprocess.check_call(["g++", "-o", exe] + [os.path.join(OUT, x) for x in
                                                ["server_driver.o", "server.o", "runtime_mock.o"]]
                          + ["-fsanitize=address,undefined"] + [f"-Wl,--wrap={f}" for f in WRAPPED]
                          + ["-L/usr/local/cuda/lib64", "-lcudart_static", "-lpthread", "-ldl", "-lrt"])
    return exe


@pytest.mark.parametrize("scenario", ["staggered", "budget", "max_resident", "bad_input", "concurrent_clients",
                                      "destroy_abandon", "destroy_drain"])
def test_server_host_logic(driver, scenario):
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=1", UBSAN_OPTIONS="halt_on_error=1")
    p = subprocess.run([driver, scenario], capture_output=True, text=True, timeout=120, env=env)
    assert p.returncode == 0 and p.stdout.strip().endswith("ok"), p.stdout + p.stderr
