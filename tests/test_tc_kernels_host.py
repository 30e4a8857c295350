"""The tcgen05 tensor-core kernels compiled for the host: one OS thread per CUDA thread under
AddressSanitizer (`tests/hostemu/cuda_host_shim.h`), the bulk copies and mbarriers on the host
model of `tests/hostemu/mbarrier_host.h`, and the tensor memory, shared-memory descriptors and
TF32 MMAs on the model of `tests/hostemu/tcgen05_host.h` (written from the PTX ISA's description
of the instructions).  The warp roles (copy producer, MMA issuer, epilogue) run as concurrent
host threads that meet only at the kernels' own mbarriers.
* `k_gemm_tc` (`csrc/gemm_tc.cu`, the batched block products of the direct interface solver):
  C = alpha A B (+ C) on operands packed by `k_pack_split`, 3xTF32 and TF32, against the FP64
  product within the error of the split.
"""
import os
import re
import shutil
import struct
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2510_25991_gb300", "csrc")
# AddressSanitizer by default; DDST_HOST_SANITIZER=thread runs the same tests under
# ThreadSanitizer, which reports accesses of two threads that no barrier orders
SANITIZE = "-fsanitize=" + os.environ.get("DDST_HOST_SANITIZER", "address")
HOSTEMU = os.path.join(ROOT, "tests", "hostemu")

# mbarrier helpers of common.cuh / umma.cuh on the host model (inside the library namespace,
# after DevStatus and set_status)
MBAR_HELPERS = r'''
inline void mbar_init(uint64_t* bar, uint32_t count) { host_mbar_init(bar, count); }
inline void fence_mbar_init() {}
inline void fence_proxy_async() { std::atomic_thread_fence(std::memory_order_seq_cst); }
inline void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) { host_mbar_arrive_expect_tx(bar, bytes); }
inline void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) { host_bulk_g2s(dst, src, bytes, bar); }
inline bool mbar_try_wait(uint64_t* bar, uint32_t parity) { return host_mbar_try_wait(bar, parity); }
inline bool mbar_wait(uint64_t* bar, uint32_t parity, DevStatus* st, int slab, int block) {
  if (host_mbar_wait(bar, parity)) return true;
  set_status(st, ST_TIMEOUT, slab, block);
  return false;
}
inline bool mbar_wait_ab(uint64_t* bar, uint32_t parity, volatile int* abort, DevStatus* st,
                         int slab, int block, long long budget = 0) {
  (void)budget;
  for (long it = 0; it < 20000000L; ++it) {
    if (host_mbar_try_wait(bar, parity)) return true;
    if (*abort) return false;
    std::this_thread::yield();
  }
  set_status(st, ST_TIMEOUT, slab, block);
  *abort = 1;
  return false;
}
'''


def _between(src, start, end):
    i = src.index(start)
    return src[i:src.index(end, i + len(start))]


def _host_tmem_calls(body):
    """The in-kernel tcgen05.alloc / relinquish / dealloc statements as calls of the model."""
    body, n1 = re.subn(r'asm volatile\("tcgen05\.alloc\.[^"]*"\s*::"r"\(\s*smem_u32\(&(\w+)\)\),\s*'
                       r'"r"\((.*?)\)\s*:\s*"memory"\);', r"host_tmem_alloc(&\1, \2);", body, flags=re.S)
    body, n2 = re.subn(r'asm volatile\("tcgen05\.relinquish_alloc_permit[^"]*"\s*:::\s*"memory"\);',
                       "host_tmem_relinquish();", body)
    body, n3 = re.subn(r'asm volatile\("tcgen05\.dealloc\.[^"]*"\s*::"r"\((\w+)\),\s*"r"\((.*?)\)'
                       r'\s*:\s*"memory"\);', r"host_tmem_dealloc(\1, \2);", body, flags=re.S)
    assert n1 == n2 == n3 >= 1 and "asm" not in body
    return body


def _common_parts():
    rd = lambda name: open(os.path.join(CSRC, name)).read()
    common, kern, umma, split = rd("common.cuh"), rd("kernels.cuh"), rd("umma.cuh"), rd("splittile.cuh")
    grab = lambda pat, src: re.search(pat, src, re.S).group(0)
    return [
        grab(r"enum PackField \{.*?\};", common),
        grab(r"struct ProbDesc \{.*?\n\};", common),
        grab(r"struct SlabDesc \{.*?\n\};", common),
        grab(r"struct DevStatus \{.*?\n\};", common),
        grab(r"enum \{ ST_SINGULAR.*?\};", common),
        grab(r"__device__ __forceinline__ void set_status\(.*?\n\}", common),
        _between(common, "template <typename T> struct Eps;", "// -----"),
        grab(r"__device__ __forceinline__ int64_t vol_index\(.*?\n\}", common),
        grab(r"struct TileDesc \{.*?\n\};", kern),
        grab(r"struct PackTask \{.*?\n\};", kern),
        grab(r"struct GemmTask \{.*?\n\};", kern),
        MBAR_HELPERS,
        grab(r"__host__ __device__ __forceinline__ uint32_t umma_off\(.*?\n\}", umma),
        grab(r"__device__ __forceinline__ uint64_t umma_desc\(.*?\n\}", umma),
        grab(r"__host__ __device__ constexpr uint32_t idesc_tf32\(.*?\n\}", umma),
        grab(r"__device__ __forceinline__ void tf32_split\(.*?\n\}", umma),
        _between(split, "constexpr int BT = 128;", "}  // namespace ddst"),
    ]


def _compile(d, name, body, main):
    cxx = shutil.which("g++")
    code = ('#include "cuda_host_shim.h"\n#include "mbarrier_host.h"\n#include "tcgen05_host.h"\n'
            "#include <cstring>\nnamespace ddst {\n" + body + "\n}  // namespace ddst\n" + main)
    (d / f"{name}.cpp").write_text(code)
    exe = d / name
    r = subprocess.run([cxx, "-std=c++20", "-O1", "-pthread", SANITIZE,
                        "-fno-omit-frame-pointer", "-I", HOSTEMU, str(d / f"{name}.cpp"), "-o",
                        str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-4000:]
    return exe


@pytest.fixture(scope="module")
def workdir(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("no host C++ compiler")
    return tmp_path_factory.mktemp("tc_host")


GEMM_MAIN = r'''
#include <fstream>
using namespace ddst;
int main(int argc, char** argv) {
  std::ifstream f(argv[1], std::ios::binary);
  int64_t h[2]; f.read((char*)h, 16);
  const int nT = (int)h[0], three = (int)h[1];
  const int64_t ld = (int64_t)nT * BT, nn = ld * ld;
  std::vector<float> A(nn), B(nn), C0(nn), C1(nn);
  f.read((char*)A.data(), 4 * nn); f.read((char*)B.data(), 4 * nn);
  f.read((char*)C0.data(), 4 * nn); C1 = C0;
  std::vector<float> Ap(2 * nn, -1.f), Bp(2 * nn, -1.f);
  std::vector<PackTask> pt = {PackTask{A.data(), Ap.data(), 0}, PackTask{B.data(), Bp.data(), 1}};
  {
    std::vector<unsigned char> sm(PACK_SMEM);
    host_smem_base = sm.data();
    host_launch2(nT * nT, 2, 256, [&] { k_pack_split(pt.data(), nT); });
  }
  std::vector<GemmTask> gt = {GemmTask{Ap.data(), Bp.data(), C0.data(), 1.0f, 0},
                              GemmTask{Ap.data(), Bp.data(), C1.data(), -0.5f, 1}};
  DevStatus st{};
  unsigned char* sm = static_cast<unsigned char*>(std::aligned_alloc(1024, (GmTc::SMEM + 1023) / 1024 * 1024));
  host_smem_base = sm;
  host_launch2(nT * nT, 2, GmTc::THREADS, [&] { k_gemm_tc(gt.data(), nT, &st, three); });
  std::free(sm);
  std::ofstream o(argv[2], std::ios::binary);
  o.write((const char*)C0.data(), 4 * nn); o.write((const char*)C1.data(), 4 * nn);
  const int32_t code = st.code; o.write((const char*)&code, 4);
  return 0;
}
'''


@pytest.fixture(scope="module")
def gemm_exe(workdir):
    src = open(os.path.join(CSRC, "gemm_tc.cu")).read()
    body = _between(src, "constexpr int PK_LS = BT + 1;", "// ---------------------------------------------------------------------------------------------\n// FMA product")
    body = body.replace("extern __shared__ float S[];", "float* S = reinterpret_cast<float*>(host_smem_base);")
    dyn = "extern __shared__ __align__(1024) unsigned char smem_raw[];"
    assert body.count(dyn) == 1
    body = _host_tmem_calls(body.replace(dyn, "unsigned char* smem_raw = host_smem_base;"))
    return _compile(workdir, "gemm_tc_host", "\n".join(_common_parts()) + "\n" + body, GEMM_MAIN)


@pytest.mark.parametrize("three", [1, 0])
def test_tensor_core_block_product_on_the_host(workdir, gemm_exe, three):
    nT = 2
    ld = nT * 128
    rng = np.random.default_rng(21 + three)
    A, B, C = (rng.standard_normal((ld, ld)).astype(np.float32) for _ in range(3))
    path = workdir / f"gemm_{three}.bin"
    path.write_bytes(struct.pack("2q", nT, three) + A.tobytes() + B.tobytes() + C.tobytes())
    out = workdir / f"gemm_{three}.out"
    r = subprocess.run([str(gemm_exe), str(path), str(out)], capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    raw = out.read_bytes()
    C0 = np.frombuffer(raw[:4 * ld * ld], dtype=np.float32).reshape(ld, ld).astype(np.float64)
    C1 = np.frombuffer(raw[4 * ld * ld:8 * ld * ld], dtype=np.float32).reshape(ld, ld).astype(np.float64)
    assert struct.unpack("i", raw[8 * ld * ld:])[0] == 0
    P = A.astype(np.float64) @ B.astype(np.float64)
    scale = np.abs(A).astype(np.float64) @ np.abs(B).astype(np.float64)
    # 3xTF32: the dropped lo*lo term and FP32 accumulation, a few 2^-22 of sum |a||b|; TF32
    # alone: operands rounded to 11 significant bits, 2^-11 each
    tol = (2.0 ** -20 if three else 2.0 ** -10) * scale
    assert np.all(np.abs(C0 - P) <= tol)
    assert np.all(np.abs(C1 - (C.astype(np.float64) - 0.5 * P)) <= 0.5 * tol + 2.0 ** -22 * np.abs(C))
