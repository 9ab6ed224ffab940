"""The boundary used from plain C: a C99 program (no Python, no PyTorch)
allocates device memory with the CUDA runtime, calls cm_create, cm_energy
and cm_solve through libcm.so, and prints the results; they must equal the
binding's on the same data."""
import os
import shutil
import subprocess

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2204_07921_gb300 as cm  # noqa: E402
import synth  # noqa: E402

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

C_SRC = r'''
#include <stdio.h>
#include <stdlib.h>
#include <cuda_runtime.h>
#include "cm.h"

int main(int argc, char** argv) {
    const int H = 48, W = 40;
    float* host = (float*)malloc(sizeof(float) * H * W);
    FILE* fp = fopen(argv[1], "rb");
    if (!fp || fread(host, sizeof(float), H * W, fp) != (size_t)(H * W)) return 10;
    fclose(fp);
    float *f = NULL, *u = NULL;
    if (cudaMalloc((void**)&f, sizeof(float) * H * W) != cudaSuccess) return 11;
    if (cudaMalloc((void**)&u, sizeof(float) * H * W) != cudaSuccess) return 12;
    cudaMemcpy(f, host, sizeof(float) * H * W, cudaMemcpyHostToDevice);
    cm_ctx* ctx = NULL;
    if (cm_create(&ctx, 0) != CM_OK) return 13;
    double E = 0.0;
    if (cm_energy(ctx, f, f, H, W, 20.0f, CM_KIND_MEAN, &E, NULL) != CM_OK) return 14;
    cm_stats st;
    if (cm_solve(ctx, f, H, W, 20.0f, CM_KIND_MEAN, 0, 5, 0.0, NULL, u, NULL, &st, NULL) != CM_OK)
        return 15;
    printf("%.17g %.17g %d\n", E, st.energy_final, st.cycles_run);
    cm_destroy(ctx);
    cudaFree(f);
    cudaFree(u);
    free(host);
    return 0;
}
'''


def test_c_program_uses_the_abi(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    cuda = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    lib = cm.build_library()
    src = tmp_path / "use_cm.c"
    src.write_text(C_SRC)
    exe = tmp_path / "use_cm"
    r = subprocess.run([cc, "-std=c99", "-O1", str(src), "-o", str(exe),
                        "-I", os.path.join(ROOT, "include"), "-I", os.path.join(cuda, "include"),
                        lib, "-L", os.path.join(cuda, "lib64"), "-lcudart",
                        "-Wl,-rpath," + os.path.dirname(lib),
                        "-Wl,-rpath," + os.path.join(cuda, "lib64")],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    img = synth.piecewise_image(48, 40, 77, 5, 0.08)
    data = tmp_path / "f.bin"
    img.f.astype(np.float32).tofile(data)
    out = subprocess.run([str(exe), str(data)], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, (out.returncode, out.stderr)
    E, Ef, n = out.stdout.split()
    fd = torch.from_numpy(img.f).cuda()
    assert float(E) == cm.cm_energy(fd, fd, 20.0, cm.MEAN)
    _, st = cm.cm_solve(fd, 20.0, cm.MEAN, cycles=5)
    assert int(n) == st.cycles_run == 5
    assert float(Ef) == st.energy_final
