"""The library's device math compiled for the host with g++ (the CUDA names it uses are replaced
by their definitions in tests/host/include) and checked against central differences: the
reverse-mode pullbacks (ProjRot3D, the S-CAM camera solve, the LM camera step, the
per-observation terms for every loss, the boundary conversions) and the Levenberg-Marquardt camera
model. No GPU is used; the
same source files are what nvcc compiles for sm_103a."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HOST = os.path.join(ROOT, "tests", "host")
FLAGS = ["-std=c++17", "-O1", "-I", os.path.join(HOST, "include"), "-D__device__=", "-D__host__=",
         "-D__forceinline__=inline", "-D__global__=inline", "-D__restrict__=", "-D__launch_bounds__(...)=",
         "-D__shared__=", "-D__align__(x)=", "-Wno-unknown-pragmas"]

# largest error of a case over its largest finite-difference component (central differences of
# step 1e-6..1e-7 in FP64 leave about 1e-8; second differences for the Hessian about 1e-9)
LIMITS = {"polar": 1e-6, "scam": 1e-5, "scam_tape": 0.0, "obs_trivial": 1e-6, "obs_huber": 1e-6,
          "obs_cauchy": 1e-6, "obs_welsch": 1e-6, "boundary": 1e-6, "lm_gradient": 1e-6, "lm_hessian": 1e-5,
          "lm_no_decrease": 0.0, "lm_adjoint": 1e-5, "lm_adjoint_steps": -12.0}


@pytest.fixture(scope="module")
def results(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not found")
    exe = str(tmp_path_factory.mktemp("device_math") / "device_math_fd")
    build = subprocess.run([gxx, *FLAGS, os.path.join(HOST, "device_math_fd.cpp"), "-o", exe],
                           capture_output=True, text=True)
    assert build.returncode == 0, build.stderr[-4000:]
    run = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert run.returncode == 0, run.stderr[-2000:]
    out = {}
    for line in run.stdout.splitlines():
        name, err, n = line.split()
        out[name] = (float(err), int(n))
    return out


@pytest.mark.parametrize("group", sorted(LIMITS))
def test_device_math_against_central_differences(results, group):
    err, n = results[group]
    assert n > 0
    assert err <= LIMITS[group], f"{group}: worst relative error {err:.3e} over {n} cases"
