"""Copy libedt's kernel sources into a build folder with the device-only
parts (inline PTX, <<<...>>> launches, dynamic shared memory) replaced by
calls into the host emulation (tests/emu/runtime.cpp).  Test infrastructure."""
import os
import re
import sys

here = os.path.dirname(os.path.abspath(__file__))
src = os.path.join(here, "../../paper_2106_03503_gb300/csrc")
out = sys.argv[1] if len(sys.argv) > 1 else os.path.join(here, "_build", "src")
os.makedirs(out, exist_ok=True)
for name in ["edt_engine.cuh", "edt_internal.h", "edt_colpass.cu", "edt_rows2d.cu", "edt_3d.cu", "edt_cityblock.cu",
             "edt_chamfer.cu", "edt_batch_table.cu"]:
    s = open(os.path.join(src, name)).read()
    s = s.replace("#include <cuda.h>", '#include "shim.h"').replace("#include <cuda_runtime.h>", '#include "shim.h"')
    s = s.replace('#include "../../include/edt.h"', '#include "edt.h"')
    s = re.sub(r'extern __shared__ __align__\(\d+\) unsigned char smem\[\];', 'unsigned char* smem = emu_smem();', s)
    # st_v8
    s = re.sub(r'asm volatile\("st\.global\.v8\.b32.*?: "memory"\);', 'emu_st_v8(q, a0, a1, a2, a3, a4, a5, a6, a7);', s, flags=re.S)
    s = re.sub(r'const uint32_t sa = \(uint32_t\)__cvta_generic_to_shared\(buf\);\s*asm volatile\("cp\.async\.bulk\.tensor.*?: "memory"\);',
               'emu_tma_store(m, buf, x, row0);', s, flags=re.S)
    s = re.sub(r'asm volatile\("(cp\.async\.bulk\.wait_group[^"]*|fence\.proxy[^"]*|cp\.async\.bulk\.commit_group;)" ::: "memory"\);', ';', s)
    s = re.sub(r'asm volatile\("bar\.sync %0, %1;" ::"r"\(id\), "r"\(nthreads\) : "memory"\);', 'emu_bar_sync(id, nthreads);', s)
    s = re.sub(r'const uint32_t da = \(uint32_t\)__cvta_generic_to_shared\(dst\);\s*asm volatile\("cp\.async\.cg\.shared\.global.*?: "memory"\);',
               'memcpy(dst, src, 16);', s, flags=re.S)
    s = re.sub(r'asm volatile\("cp\.async\.commit_group;\\n\\tcp\.async\.wait_group 0;" ::: "memory"\);', ';', s)
    # launches
    def split_top(t):
        parts, depth, cur = [], 0, ""
        for ch in t:
            if ch == "(":
                depth += 1
            elif ch == ")":
                depth -= 1
            if ch == "," and depth == 0:
                parts.append(cur); cur = ""
            else:
                cur += ch
        parts.append(cur)
        return parts
    def launch(m):
        cfg = split_top(m.group(2))
        return f'emu_launch({cfg[0]}, {cfg[1]}, {cfg[2] if len(cfg) > 2 else "0"}, [=]() {{ {m.group(1)}({m.group(3)}); }});'
    s = re.sub(r'(\b[\w:]+(?:<[^<>;]*>)?)<<<(.*?)>>>\((.*?)\);', launch, s, flags=re.S)
    left = [ln for ln in s.splitlines() if "asm volatile" in ln or "<<<" in ln]
    assert not left, (name, left)
    open(os.path.join(out, name), "w").write(s)

