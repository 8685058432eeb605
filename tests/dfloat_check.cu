// Host driver for tests/test_dfloat_host.py: reads operands (C99 hex floats), prints the
// double-float results of csrc/dfloat.cuh (a host build of the inline functions the kernels use).
//   c v                  dfl(v) from a double
//   a|s|m ah al bh bl    (ah + al) + - * (bh + bl)
//   f ah al b            (ah + al) * b, b an FP32 number
//   x ah al b xh xl      (ah + al) + b * (xh + xl), the band-product accumulation
//   A k [b xh xl]*k      sum of k products b * (xh + xl) in the lazily normalised accumulator
//   d ah al bh bl ch cl dh dl   (ah + al)(bh + bl) + (ch + cl)(dh + dl), one normalisation
#include <cstdio>
#include "dfloat.cuh"

using fk::dfl;

int main() {
    char op[8];
    while (scanf("%7s", op) == 1) {
        dfl r;
        if (op[0] == 'c') {
            double v;
            if (scanf("%la", &v) != 1) return 1;
            r = dfl(v);
        } else if (op[0] == 'f') {
            float ah, al, b;
            if (scanf("%a %a %a", &ah, &al, &b) != 3) return 1;
            r = fk::df_mul_f(dfl(ah, al), b);
        } else if (op[0] == 'A') {
            int k;
            if (scanf("%d", &k) != 1) return 1;
            fk::dacc acc;
            fk::dacc_zero(acc);
            for (int i = 0; i < k; ++i) {
                float b, xh, xl;
                if (scanf("%a %a %a", &b, &xh, &xl) != 3) return 1;
                fk::dacc_add_fx(acc, b, dfl(xh, xl));
            }
            r = fk::dacc_value(acc);
        } else if (op[0] == 'd') {
            float v[8];
            for (int i = 0; i < 8; ++i)
                if (scanf("%a", &v[i]) != 1) return 1;
            r = fk::df_dot2(dfl(v[0], v[1]), dfl(v[2], v[3]), dfl(v[4], v[5]), dfl(v[6], v[7]));
        } else if (op[0] == 'x') {
            float ah, al, b, xh, xl;
            if (scanf("%a %a %a %a %a", &ah, &al, &b, &xh, &xl) != 5) return 1;
            r = dfl(ah, al);
            fk::df_acc_fx(r, b, dfl(xh, xl));
        } else {
            float ah, al, bh, bl;
            if (scanf("%a %a %a %a", &ah, &al, &bh, &bl) != 4) return 1;
            const dfl a(ah, al), b(bh, bl);
            if (op[0] == 'a') r = a + b;
            else if (op[0] == 's') r = a - b;
            else if (op[0] == 'm') r = a * b;
            else return 2;
        }
        printf("%a %a\n", r.hi, r.lo);
    }
    return 0;
}
