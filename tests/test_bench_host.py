"""Host-side logic of bench.py that needs no GPU: the hash that ties the committed DRAM traffic
to the seeding kernels' code."""
import bench


def test_kernel_hash_ignores_comments_and_blank_lines():
    src = '''// a comment
#include "x.h"   /* a block
comment */
int f(int a) {  // trailing
    const char *s = "// not a comment /* nor this */";

    return a + '/';
}
'''
    same = '''#include "x.h"
int f(int a) {
    const char *s = "// not a comment /* nor this */";
    return a + '/';
}'''
    assert bench.strip_comments(src) == same
    assert bench.strip_comments(src.replace("return a + '/'", "return a - '/'")) != same

